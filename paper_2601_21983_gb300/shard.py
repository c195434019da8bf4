"""Particle-sharded sampler across ranks: one libsmc context per rank (one GPU
each) holds a consecutive range of the J particles, the training data is
replicated, and the ranks exchange what the method couples (Sec. 2):

* after every move, the raw log-weights (J doubles, all-gather): each rank
  normalises all J with the library's kernel (eqs. normalise, jeff), so every
  rank holds the same w~ and ESS;
* SDA's weighted moments (Sec. 3.1): each rank's partial sums, all-gathered
  and added in rank order;
* resampling (when ESS < J/2): every rank draws the same uniforms from its
  context's stream and computes the same ancestors with the library's kernel;
  then each particle row travels from the rank holding its ancestor to the
  rank that holds its slot (one all-to-all).

A context's particle j draws the prior and momentum streams of global particle
first + j (smc_set_shard), so G ranks reproduce the single-context run.

The collective is torch.distributed on host tensors (gloo) or device tensors
(NCCL); the exchange logic itself (`Layout`, `exchange_plan`, `exchange_rows`)
does no arithmetic on the particles and is tested with gloo ranks on CPU.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Layout:
    """J particles over `world` ranks in consecutive ranges of J // world."""
    J: int
    world: int

    def __post_init__(self):
        if self.world < 1 or self.J % self.world != 0:
            raise ValueError(f"J = {self.J} must be a multiple of the number of ranks ({self.world})")

    @property
    def per_rank(self) -> int:
        return self.J // self.world

    def first(self, rank: int) -> int:
        return rank * self.per_rank

    def owner(self, g):
        return np.asarray(g) // self.per_rank


def exchange_plan(anc, layout: Layout, rank: int):
    """Rows to send and slots to fill for this rank after resampling with global
    ancestors `anc` [J] (new particle g takes the state of old particle anc[g]).

    Returns (send_rows, send_counts, recv_slots, recv_counts): this rank sends
    its local rows send_rows (grouped by destination rank, destinations in rank
    order, and within a destination in increasing slot order), send_counts[d]
    of them to rank d; it receives recv_counts[s] rows from rank s, which fill
    its local slots recv_slots (grouped by source rank in rank order, slots
    increasing within a source)."""
    anc = np.asarray(anc, dtype=np.int64)
    n, w = layout.per_rank, layout.world
    src = layout.owner(anc)                                   # rank holding each ancestor
    send_rows, send_counts = [], np.zeros(w, np.int64)
    for d in range(w):
        g = np.arange(layout.first(d), layout.first(d) + n)  # destination slots of rank d
        mine = src[g] == rank
        send_rows.append(anc[g[mine]] - layout.first(rank))
        send_counts[d] = int(mine.sum())
    my = np.arange(layout.first(rank), layout.first(rank) + n)
    recv_slots, recv_counts = [], np.zeros(w, np.int64)
    for s in range(w):
        sel = np.nonzero(src[my] == s)[0]
        recv_slots.append(sel)
        recv_counts[s] = len(sel)
    return (np.concatenate(send_rows).astype(np.int64), send_counts,
            np.concatenate(recv_slots).astype(np.int64), recv_counts)


def exchange_rows(rows, anc, layout: Layout, rank: int, group=None):
    """Resampled local rows: out[i] = old row of global particle anc[first + i].
    `rows` is this rank's [per_rank, W] tensor (host for gloo, device for NCCL)."""
    import torch
    import torch.distributed as dist

    send_rows, send_counts, recv_slots, recv_counts = exchange_plan(anc, layout, rank)
    idx = torch.from_numpy(send_rows).to(rows.device)
    send = rows.index_select(0, idx).contiguous()
    recv = torch.empty((int(recv_counts.sum()),) + tuple(rows.shape[1:]), dtype=rows.dtype, device=rows.device)
    if layout.world == 1:
        recv.copy_(send)
    else:
        dist.all_to_all_single(recv, send, output_split_sizes=[int(x) for x in recv_counts],
                               input_split_sizes=[int(x) for x in send_counts], group=group)
    out = torch.empty_like(rows)
    out[torch.from_numpy(recv_slots).to(rows.device)] = recv
    return out


def all_gather_cat(x, group=None):
    """Concatenate every rank's 1-D tensor `x` in rank order."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        return x.clone()
    parts = [torch.empty_like(x) for _ in range(world)]
    dist.all_gather(parts, x, group=group)
    return torch.cat(parts)


class ShardedSampler:
    """The SMC sampler with its J particles spread over the ranks of a process
    group (one context per rank on the current CUDA device).  Methods mirror
    the ABI: set_schedule, anneal_next, resample, step, predict; every rank
    calls them in the same order.  The learned proposal's features are global
    statistics of the particles and are not sharded: step() takes the plain
    proposal only."""

    def __init__(self, model, X, J, cfg, y_class=None, y_value=None, group=None):
        import torch
        import torch.distributed as dist

        from . import smc as S

        self.S = S
        self.group = group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.layout = Layout(J, self.world)
        self.J = J
        self.n = self.layout.per_rank
        # collectives go through host tensors on gloo and device tensors otherwise
        self.dev = torch.device("cpu")
        if dist.is_initialized() and dist.get_backend(group) != "gloo":
            self.dev = torch.device("cuda", torch.cuda.current_device())
        cfg.n_particles = self.n
        self.resampler = cfg.resampler
        self.ctx = S.smc_init(model, X, y_class=y_class, y_value=y_value, cfg=cfg)
        S.smc_set_shard(self.ctx, self.layout.first(self.rank))
        self.D = S.smc_num_params(self.ctx)
        self.ess = float(J)
        self.wn = np.full(J, 1.0 / J)
        self.stream = torch.cuda.current_stream()

    # ------------------------------------------------------------- helpers
    def _gather_host(self, a):
        import torch
        t = torch.from_numpy(np.ascontiguousarray(a)).to(self.dev)
        return all_gather_cat(t, self.group).cpu().numpy()

    def _normalise_global(self):
        """All-gather the raw log-weights and normalise all J of them on this
        rank's GPU; install this rank's slice and the global ESS."""
        import torch
        S = self.S
        _, logw, _ = S.smc_get_state(self.ctx, self.n, self.D, theta=False)
        allw = torch.from_numpy(self._gather_host(logw)).cuda()
        wn = torch.empty_like(allw)
        ess = torch.empty(1, dtype=torch.float64, device="cuda")
        S.smc_k_normalise(allw, wn, ess, self.stream)
        torch.cuda.synchronize()
        self.wn = wn.cpu().numpy()
        self.ess = float(ess.item())
        f = self.layout.first(self.rank)
        S.smc_set_weights(self.ctx, self.wn[f:f + self.n], self.ess)
        return self.ess

    # ------------------------------------------------------------- the iteration
    def set_schedule(self, sched):
        self.S.smc_set_schedule(self.ctx, sched)
        return self._normalise_global()

    def anneal_next(self):
        S = self.S
        part = S.smc_sda_partials(self.ctx)            # zeros are harmless for fixed schedules
        allp = self._gather_host(part).reshape(self.world, 4)
        m = np.zeros(4)
        for r in range(self.world):                    # fixed order: identical on every rank
            m += allp[r]
        return S.smc_anneal_next_moments(self.ctx, m)

    def resample(self, force=False):
        """Resample when the global ESS < J/2 (or when forced); returns whether
        it did and the global ancestors."""
        import torch
        S = self.S
        if not force and not (self.ess < 0.5 * self.J):
            return False, None
        kind = self.resampler
        nu = 1 if kind == S.RESAMPLE_SYSTEMATIC else self.J
        u = S.smc_draw_uniforms(self.ctx, nu)
        wn = torch.from_numpy(self.wn).cuda()
        anc_d = torch.empty(self.J, dtype=torch.int32, device="cuda")
        S.smc_k_resample(wn, kind, u, anc_d, self.stream)
        torch.cuda.synchronize()
        anc = anc_d.cpu().numpy().astype(np.int64)
        theta, _, logpi = S.smc_get_state(self.ctx, self.n, self.D)
        theta_new = exchange_rows(torch.from_numpy(theta).to(self.dev), anc, self.layout, self.rank,
                                  self.group).cpu().numpy()
        logpi_new = exchange_rows(torch.from_numpy(logpi.reshape(self.n, 1)).to(self.dev), anc, self.layout,
                                  self.rank, self.group).cpu().numpy().reshape(self.n)
        # -log J computed on the GPU, as the single-context resampling writes it
        logw_new = (-torch.log(torch.full((self.n,), float(self.J), dtype=torch.float64, device="cuda"))).cpu().numpy()
        S.smc_set_state(self.ctx, np.ascontiguousarray(theta_new), logw_new, logpi_new)
        self.wn = np.full(self.J, 1.0 / self.J)
        self.ess = float(self.J)
        f = self.layout.first(self.rank)
        S.smc_set_weights(self.ctx, self.wn[f:f + self.n], self.ess)
        return True, anc

    def step(self, h, S_steps):
        st = self.S.smc_step(self.ctx, h, S_steps, self.S.PROPOSAL_PLAIN)
        st["ess"] = self._normalise_global()
        return st

    def predict(self, x, n_classes):
        """Posterior predictive over all J particles: each rank's weighted sum of
        its particles' softmax outputs, added over ranks in rank order."""
        part = self.S.smc_posterior_predict(self.ctx, x, np.empty((x.shape[0], n_classes), np.float32))
        allp = self._gather_host(part.reshape(-1)).reshape((self.world,) + part.shape)
        out = np.zeros(part.shape, np.float64)
        for r in range(self.world):
            out += allp[r]
        return out

    def state(self):
        """This rank's particles, raw log-weights and log pi."""
        return self.S.smc_get_state(self.ctx, self.n, self.D)

    def close(self):
        self.S.smc_destroy(self.ctx)

"""CPU tests of the particle-sharded exchange (no GPU): the routing plan that
moves particle rows between ranks after resampling, checked against the
definition new[g] = old[anc[g]], and the same exchange run through gloo ranks
(world sizes 2 and 3) on CPU tensors, including the all-gather of per-rank
vectors in rank order."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2601_21983_gb300.shard import Layout, all_gather_cat, exchange_plan, exchange_rows  # noqa: E402

ANCESTOR_CASES = {
    "random": lambda J, r: r.integers(0, J, J),
    "identity": lambda J, r: np.arange(J),
    "one_parent": lambda J, r: np.full(J, J - 1),
    "reversed": lambda J, r: np.arange(J)[::-1].copy(),
    "sorted_systematic": lambda J, r: np.sort(r.integers(0, J, J)),
}


def _simulate(anc, layout):
    """Run every rank's plan by hand and assemble the result."""
    J, n = layout.J, layout.per_rank
    old = np.arange(J) * 10 + 7                       # a value that identifies each old particle
    plans = [exchange_plan(anc, layout, r) for r in range(layout.world)]
    out = np.full(J, -1)
    for d in range(layout.world):
        pieces = []
        for s in range(layout.world):
            send_rows, send_counts, _, _ = plans[s]
            start = int(send_counts[:d].sum())
            rows = send_rows[start:start + int(send_counts[d])] + layout.first(s)
            pieces.append(old[rows])
        recv = np.concatenate(pieces)
        _, _, recv_slots, recv_counts = plans[d]
        assert len(recv) == len(recv_slots) == int(recv_counts.sum())
        out[layout.first(d) + recv_slots] = recv
    return old, out


@pytest.mark.parametrize("J,world", [(8, 1), (12, 2), (12, 3), (32, 4), (30, 5)])
@pytest.mark.parametrize("case", sorted(ANCESTOR_CASES))
def test_plan_matches_definition(J, world, case):
    r = np.random.default_rng(J * 31 + world)
    anc = ANCESTOR_CASES[case](J, r)
    layout = Layout(J, world)
    old, out = _simulate(anc, layout)
    assert np.array_equal(out, old[anc])
    # what rank s sends to d is what d expects from s
    plans = [exchange_plan(anc, layout, q) for q in range(world)]
    for s in range(world):
        for d in range(world):
            assert plans[s][1][d] == plans[d][3][s]


def test_layout_rejects_uneven_split():
    with pytest.raises(ValueError):
        Layout(10, 3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, J, seeds, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        layout = Layout(J, world)
        n = layout.per_rank
        D = 5
        full = torch.arange(J * D, dtype=torch.float32).reshape(J, D) + 0.25
        gathered = all_gather_cat(torch.arange(n, dtype=torch.float64) + 100.0 * rank)
        expect = torch.cat([torch.arange(n, dtype=torch.float64) + 100.0 * q for q in range(world)])
        ok = bool(torch.equal(gathered, expect))
        for seed in seeds:
            anc = np.random.default_rng(seed).integers(0, J, J)
            mine = full[layout.first(rank):layout.first(rank) + n].clone()
            got = exchange_rows(mine, anc, layout, rank)
            want = full[torch.from_numpy(anc[layout.first(rank):layout.first(rank) + n])]
            ok = ok and bool(torch.equal(got, want))
        with open(os.path.join(out_dir, f"rank{rank}.ok"), "w") as f:
            f.write("1" if ok else "0")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,J", [(2, 16), (3, 12)])
def test_exchange_through_gloo_ranks(tmp_path, world, J):
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, J, [1, 2, 3], str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        assert (tmp_path / f"rank{r}.ok").read_text() == "1", r

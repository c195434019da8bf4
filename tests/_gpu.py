"""Helpers shared by the GPU tests: build a sampler context through the C ABI
and the matching oracle sampler on the same seeded inputs."""
import numpy as np

from oracle import nn, rng, smc as osmc
from paper_2601_21983_gb300 import smc as S

ACT = {nn.TANH: S.ACT_TANH, nn.RELU: S.ACT_RELU, nn.IDENTITY: S.ACT_IDENTITY}


def make_pair(spec, X, y, J, seed, precision=S.PREC_FP32, chunk=0, scaled=True, prior_sigma=1.0,
              resampler=S.RESAMPLE_SYSTEMATIC, stream=None, timing=0):
    """(ctx, oracle Sampler) on the same data, particles drawn by `synthetic`."""
    import torch
    lik = S.LIK_CATEGORICAL if spec.likelihood == nn.CATEGORICAL else S.LIK_GAUSSIAN
    model = S.make_model(spec.layers, spec.input_shape, ACT[spec.activation], lik, prior_sigma, spec.noise_sigma)
    cfg = S.make_config(J, seed, precision, resampler, 1 if scaled else 0, chunk,
                        stream if stream is not None else torch.cuda.current_stream(), timing)
    X = np.ascontiguousarray(X, np.float32)
    if lik == S.LIK_CATEGORICAL:
        ctx = S.smc_init(model, X, y_class=np.ascontiguousarray(y, np.int32), cfg=cfg)
    else:
        ctx = S.smc_init(model, X, y_value=np.ascontiguousarray(y, np.float32), cfg=cfg)
    perm = rng.fisher_yates_permutation(X.shape[0], seed)
    orc = osmc.Sampler(spec, X, y, J, perm, prior_sigma=prior_sigma, scaled=scaled)
    return ctx, orc, model


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_eval(orc):
    """log pi, LL gradient (prior excluded), La, Lb per particle at orc.theta."""
    J = orc.J
    lp, la, lb = np.empty(J), np.empty(J), np.empty(J)
    g = np.empty((J, orc.D))
    for j in range(J):
        lp[j], gg, la[j], lb[j] = orc.target(orc.theta[j])
        g[j] = gg + orc.theta[j] / orc.sigma ** 2
    return lp, g, la, lb

"""GPU tests of the stateless kernels, called through the C ABI: Philox draws
(bit-exact against the oracle's Philox), the tcgen05/TMA GEMM (against a plain
PyTorch fp32 matmul of the same BF16 operands), FP64 normalisation / ESS and
the fixed-point resampler (bit-exact ancestors on identical weights)."""
import numpy as np
import pytest

import synthetic
from oracle import rng, smc as osmc

torch = pytest.importorskip("torch")
from paper_2601_21983_gb300 import smc as S  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    S.load()


def test_philox_u32_bitexact():
    n = 4096
    for key, c2, c3 in [((0, 0), 0, 0), ((0xA4093822, 0x299F31D0), 7, 2), ((0xFFFFFFFF, 0x12345678), 99, 1)]:
        out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
        S.smc_k_philox_u32(key[0], key[1], c2, c3, out)
        got = out.cpu().numpy().view(np.uint32)
        for q in [0, 1, 2, 3, 1000, n - 1]:
            assert tuple(int(v) for v in got[q]) == rng.philox4x32_10((q, 0, c2, c3), key)


def test_philox_normals_match_oracle():
    for seed, sid, it, off, n in [(1, 2, 0, 0, 1001), (0xDEADBEEF12345, 2, 7, 13, 517)]:
        out = torch.empty(n, dtype=torch.float32, device="cuda")
        S.smc_k_philox_normals(seed, sid, it, off, out)
        ref = rng.philox_normals(seed, sid, it, n, offset=off)
        got = out.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref)) < 2e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 200, 100), (5, 17, 16), (513, 1024, 784),
                                   (1000, 785, 700), (129, 400, 1000), (64, 800, 48)])
def test_tcgen05_gemm_matches_fp32_reference(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N)
    Kp = (K + 7) // 8 * 8
    A = torch.randn(M, Kp, device="cuda", generator=g).to(torch.bfloat16)[:, :K]
    B = torch.randn(N, Kp, device="cuda", generator=g).to(torch.bfloat16)[:, :K]
    C = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
    S.smc_k_gemm_bf16(A, B, C)
    torch.cuda.synchronize()
    ref = A.float() @ B.float().T
    err = (C - ref).abs().max().item()
    assert err <= 1e-4 * ref.abs().max().item() + 1e-4, err
    # accumulate mode adds a second product
    S.smc_k_gemm_bf16(A, B, C, accumulate=True)
    torch.cuda.synchronize()
    assert (C - 2 * ref).abs().max().item() <= 2e-4 * ref.abs().max().item() + 2e-4


def _store(L, mn_major, kind):
    """Lay the logical operands L [batch][rows][K] (BF16) out in device memory:
    kind "dense" (one matrix after another), "interleaved" (batches side by side
    inside each row, as in a [rows][J][H] activation array) or "shared" (one
    matrix, batch stride 0).  Row padding is NaN, so a read past the logical
    extent would poison the product.  Returns (buffer, (mn_major, ld, bstride))."""
    nb, rows, K = L.shape
    inner, outer = (rows, K) if mn_major else (K, rows)
    X = L.transpose(1, 2) if mn_major else L                     # [batch][outer][inner]
    ld = (inner + 7) // 8 * 8 + 8
    if kind == "interleaved":
        buf = torch.full((outer, nb, ld), float("nan"), device="cuda", dtype=torch.bfloat16)
        buf[:, :, :inner] = X.permute(1, 0, 2)
        return buf.reshape(-1), (mn_major, nb * ld, ld)
    buf = torch.full((nb, outer, ld), float("nan"), device="cuda", dtype=torch.bfloat16)
    buf[:, :, :inner] = X
    return buf.reshape(-1), (mn_major, ld, 0 if kind == "shared" else outer * ld)


@pytest.mark.parametrize("M,N,K,batch,a,b", [
    (300, 200, 100, 3, (0, "dense"), (0, "dense")),
    (257, 401, 200, 2, (1, "dense"), (1, "dense")),
    (400, 401, 1000, 4, (1, "interleaved"), (1, "interleaved")),   # weight gradient of a hidden layer
    (1000, 400, 400, 3, (0, "interleaved"), (0, "dense")),         # forward of a hidden layer
    (1000, 400, 400, 3, (0, "interleaved"), (1, "dense")),         # adjoint through a hidden layer
    (600, 785, 300, 1, (1, "dense"), (0, "dense")),                # first-layer weight gradient
    (130, 64, 17, 2, (0, "shared"), (1, "dense")),
    (64, 16, 8, 5, (1, "dense"), (0, "shared")),
    (256, 128, 64, 64, (0, "dense"), (1, "interleaved")),
])
def test_batched_tcgen05_gemm_matches_fp32_reference(M, N, K, batch, a, b):
    """smc_k_gemm_bf16_batched (CTA-pair tcgen05, K-major and MN-major operands)
    against a plain PyTorch fp32 matmul of the same BF16 operands, per batch."""
    g = torch.Generator(device="cuda").manual_seed(M + 3 * N + 7 * K + batch)
    LA = torch.randn(1 if a[1] == "shared" else batch, M, K, device="cuda", generator=g).to(torch.bfloat16)
    LB = torch.randn(1 if b[1] == "shared" else batch, N, K, device="cuda", generator=g).to(torch.bfloat16)
    bufA, la = _store(LA, a[0], a[1])
    bufB, lb = _store(LB, b[0], b[1])
    ldc = N + 3
    C = torch.full((batch, M, ldc), float("nan"), device="cuda", dtype=torch.float32)
    S.smc_k_gemm_bf16_batched(bufA, la, bufB, lb, C.reshape(-1), (ldc, M * ldc), M, N, K, batch)
    torch.cuda.synchronize()
    ref = LA.float().expand(batch, M, K) @ LB.float().expand(batch, N, K).transpose(1, 2)
    got = C[:, :, :N]
    err = (got - ref).abs().max().item()
    assert err <= 1e-4 * ref.abs().max().item() + 1e-4, err
    assert torch.isnan(C[:, :, N:]).all()          # columns past N untouched
    S.smc_k_gemm_bf16_batched(bufA, la, bufB, lb, C.reshape(-1), (ldc, M * ldc), M, N, K, batch, accumulate=True)
    torch.cuda.synchronize()
    assert (C[:, :, :N] - 2 * ref).abs().max().item() <= 2e-4 * ref.abs().max().item() + 2e-4


def test_normalise_matches_oracle():
    r = np.random.default_rng(0)
    for J in [1, 5, 256, 1024, 4096]:
        logw = r.normal(scale=30.0, size=J)
        if J > 4:
            logw[3] = -np.inf
        lw = torch.tensor(logw, device="cuda", dtype=torch.float64)
        wn = torch.empty(J, device="cuda", dtype=torch.float64)
        ess = torch.empty(1, device="cuda", dtype=torch.float64)
        S.smc_k_normalise(lw, wn, ess)
        ref = osmc.normalise(logw)
        assert np.allclose(wn.cpu().numpy(), ref, rtol=1e-12, atol=1e-300)
        assert abs(ess.item() - osmc.ess(ref)) <= 1e-10 * osmc.ess(ref)


@pytest.mark.parametrize("J", [1, 2, 7, 256, 1000, 1024, 4096])
def test_resampling_bitexact(J):
    for trial in range(4):
        wn = synthetic.normalised_weights(J, 17 * J + trial, spread=[0.5, 2.0, 4.0, 8.0][trial])
        u = synthetic.uniforms(J, 5 * J + trial)
        wd = torch.tensor(wn, device="cuda", dtype=torch.float64)
        anc = torch.empty(J, device="cuda", dtype=torch.int32)
        S.smc_k_resample(wd, S.RESAMPLE_SYSTEMATIC, u[:1], anc)
        assert np.array_equal(anc.cpu().numpy(), osmc.systematic_ancestors(wn, float(u[0])))
        S.smc_k_resample(wd, S.RESAMPLE_MULTINOMIAL, u, anc)
        assert np.array_equal(anc.cpu().numpy(), osmc.multinomial_ancestors(wn, u))


def test_resampling_degenerate_weights():
    J = 64
    for wn in [np.eye(J)[5], np.full(J, 1.0 / J), np.eye(J)[J - 1]]:
        wd = torch.tensor(wn, device="cuda", dtype=torch.float64)
        anc = torch.empty(J, device="cuda", dtype=torch.int32)
        for u in [0.0, 0.5, np.nextafter(1.0, 0.0)]:
            S.smc_k_resample(wd, S.RESAMPLE_SYSTEMATIC, [u], anc)
            assert np.array_equal(anc.cpu().numpy(), osmc.systematic_ancestors(wn, u))

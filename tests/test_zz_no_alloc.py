"""The allocation-free resampling entry point (smc_k_resample_noalloc),
called through the C ABI, must return the same ancestors as smc_k_resample
on consecutive calls.  It exists for callers that cannot allocate device
memory (code under an allocator that owns all device memory, loops that
cannot take the device-wide synchronisation of cudaFree).  This
file is collected last so a failure here leaves every other test already run;
it passes alone in a fresh process as well."""
import numpy as np
import pytest

import synthetic

torch = pytest.importorskip("torch")
from paper_2601_21983_gb300 import smc as S  # noqa: E402

pytestmark = pytest.mark.gpu


def _both(wn, kind, u):
    wd = torch.tensor(wn, device="cuda", dtype=torch.float64)
    a_ref = torch.empty(len(wn), device="cuda", dtype=torch.int32)
    a_new = torch.full((len(wn),), -1, device="cuda", dtype=torch.int32)
    S.smc_k_resample(wd, kind, u, a_ref)
    S.smc_k_resample_noalloc(wd, kind, u, a_new)
    return a_ref.cpu().numpy(), a_new.cpu().numpy()


@pytest.mark.parametrize("kind", [S.RESAMPLE_SYSTEMATIC, S.RESAMPLE_MULTINOMIAL])
def test_noalloc_matches_existing_entry_on_consecutive_calls(kind):
    S.load()
    # two calls in a row with different sizes and draws: the second call must not
    # see anything of the first one's scratch contents
    for J, seed in [(4096, 1), (37, 2)]:
        wn = synthetic.normalised_weights(J, seed, spread=3.0)
        u = synthetic.uniforms(J, 100 + seed)
        ref, new = _both(wn, kind, u if kind == S.RESAMPLE_MULTINOMIAL else u[:1])
        assert np.array_equal(ref, new)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    S.load()
    wd = torch.full((4097,), 1.0 / 4097, device="cuda", dtype=torch.float64)
    anc = torch.empty(4097, device="cuda", dtype=torch.int32)
    with pytest.raises(S.SMCError) as e:
        S.smc_k_resample_noalloc(wd, S.RESAMPLE_SYSTEMATIC, [0.5], anc)
    assert e.value.status == 1 and "4096" in str(e.value)

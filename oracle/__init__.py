"""FP64 CPU oracle for the data-annealed SMC sampler of "Investigating Batch
Inference in a Sequential Monte Carlo Framework for Neural Networks".

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` use it.  It shares no
code with the CUDA library (`paper_2601_21983_gb300/`), and neither imports the
other; the only module both sides use is `synthetic`, which draws input data
and holds none of the method's arithmetic.

The oracle is plain, slow and written for checking by eye against the paper:
numpy in float64, one particle at a time, library primitives (matmul, einsum,
cumsum, sort) as single steps and nothing blocked, fused or reordered.

Modules and the passages they follow:
  rng        counter-based generators used by the method (SplitMix64, Philox4x32-10,
             Box-Muller) and the Fisher-Yates draw of mini-batch order (Sec. 3:
             mini-batches drawn without replacement).
  schedules  the five fixed data-annealing schedules (Sec. 3.1) and the smooth
             data-annealing (SDA) temperature rule (Sec. 3.1, eqs. beta_initial_data_k,
             beta_annealed_k and the weighted moments that follow them).
  nn         network log-likelihoods and their gradients (Sec. 2 target, Sec. 3
             eq. approx-grad), plus the linear-Gaussian model with a closed-form
             posterior used to pin the sampler.
  smc        the sampler: initial weights (eq. init_weight), leapfrog move
             (eqs. mom_first, pos_update, mom_second), weight update with the
             reversed-momentum L-kernel (eq. weight_update_fp), normalisation
             (eq. normalise), ESS (eq. jeff), resampling and the weighted
             posterior estimate.
  learned    the learned per-layer preconditioner/step proposal (not in the paper;
             a generalisation of the leapfrog kernel to a diagonal mass matrix).

Every function states the passage it follows.  Readings taken where the paper
is silent or ambiguous are listed in the repository's design notes and named
in the docstrings ("reading r<n>").
"""

"""Element-wise parity of the kernels the served BF16 path runs (and the
benchmark times) with the FP64 oracle, each kernel on its own.

The BF16 path computes the AEV and the forces in FP32 with the hardware
approximations (ex2, lg2, rcp, rsqrt .approx) and stores every AEV row as a
BF16 pair, G_hi + G_lo, where G_lo is the BF16 rounding of G - G_hi. The
network consumes that pair, so the test compares G_hi + G_lo with the
oracle's AEV (section "Optimization Through NNPOps": the atom-centered
symmetry functions), and runs the force kernel alone on a fixed dE/dG
(section "PyTorch Model Support": forces by backpropagation), so that its
error is not hidden behind the network's BF16 rounding.

Tolerances (derived, not fitted):
* AEV: the FP32 bar of the accurate path, |dG| <= 2e-5 max(1, |G|) per
  element (FP32 geometry, whose r error ~2^-23 r moves a Gaussian term by at
  most 0.25 sqrt(2 eta / e) dr; the .approx functions add ~2^-22 relative per
  term), plus the BF16-pair representation error 2^-16 |G| (G_lo is exact to
  half an ulp of its own 8-bit significand: 2^-9 * 2^-8 relative to G; the
  bound is taken twice for safety). Structural zeros (absent element pairs)
  are exactly zero on both sides.
* Split structure: |G_lo| <= half an ulp of G_hi in BF16 (G_hi is the BF16
  rounding of the FP32 value).
* Forces from a fixed dE/dG: max |dF| <= 1e-4 eV/A, the FP32 force bar of the
  path, applied to the force kernel alone. dE/dG is rounded to BF16 before
  both sides see it (the BF16 path stores dE/dG in BF16), so the comparison
  isolates the kernel's arithmetic.
"""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu

AEV_ABS = 2e-5
AEV_PAIR_REL = 2.0 ** -16
F_MAX = 1e-4


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_2310_03121_b300 as P

    P.load()
    return P


@pytest.fixture(scope="module")
def wts():
    return gen.make_weights()


@pytest.fixture(scope="module")
def W(P, wts):
    return P.Weights(wts)


@pytest.fixture(scope="module")
def OW(wts):
    return oracle.Weights(wts)


CASES = {
    "config0": lambda: gen.make_config(0),
    "config1": lambda: gen.make_config(1),
    "box300": lambda: gen.random_molecule(300, seed=21, density=0.1, periodic=True),
    "config4": lambda: gen.make_config(4),
}


def _bf16(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _rows(c):
    """Rows checked: all of them, or a seeded sample of 400 for the 21,080-atom box."""
    if c.n <= 2000:
        return np.arange(c.n)
    return np.sort(np.random.default_rng(9).choice(c.n, 400, replace=False))


@pytest.mark.parametrize("case", list(CASES))
def test_fast_aev_pair_matches_oracle(P, W, case):
    c = CASES[case]()
    s = P.System(W, c.species, c.coords, c.cell, precision="bf16")
    s.energy_forces()
    hi, lo = s.debug_aev_split()
    G = s.debug_aev()
    assert np.array_equal(G, hi + lo)
    rows = _rows(c)
    ref = oracle.aev_subset(c.species, c.coords, c.cell, rows) if rows.size < c.n else oracle.aev(c.species, c.coords,
                                                                                                    c.cell)
    got = G[rows].astype(np.float64)
    err = np.abs(got - ref)
    bound = AEV_ABS * np.maximum(1.0, np.abs(ref)) + AEV_PAIR_REL * np.abs(ref)
    worst = np.unravel_index(np.argmax(err / bound), err.shape)
    assert (err <= bound).all(), (case, worst, got[worst], ref[worst], float(err.max()))
    assert (got[ref == 0.0] == 0.0).all()                       # absent terms stay exactly zero
    # the split: G_hi is the BF16 rounding of the FP32 value, G_lo the rest
    h, l = hi[rows].astype(np.float64), lo[rows].astype(np.float64)
    assert np.array_equal(_bf16(h), h) and np.array_equal(_bf16(l), l)
    nz = h != 0.0
    ulp = 2.0 ** (np.floor(np.log2(np.abs(h[nz]))) - 7)
    assert (np.abs(l[nz]) <= 0.5 * ulp).all()
    assert (l[~nz] == 0.0).all()
    print(f"{case}: fast AEV max |dG| = {err.max():.3e}, max |dG|/max(1,|G|) = "
          f"{(err / np.maximum(1.0, np.abs(ref))).max():.3e}")
    s.close()


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
def test_force_kernel_alone_matches_oracle(P, W, OW, case, precision):
    c = CASES[case]()
    s = P.System(W, c.species, c.coords, c.cell, precision=precision)
    s.energy_forces()
    if c.n <= 2000:
        _, g = oracle.aev_grad(c.species, c.coords, c.cell, OW)      # the network's own dE/dG
    else:
        g = np.random.default_rng(4).normal(size=(c.n, oracle.AEV_LEN)) * 0.03   # its scale, every column
    g = _bf16(g) if precision == "bf16" else g.astype(np.float32).astype(np.float64)
    F = s.debug_forces(g)
    F_ref = oracle.forces_from_dEdG(c.species, c.coords, c.cell, g)
    err = np.abs(F - F_ref)
    print(f"{case} {precision}: force kernel max |dF| = {err.max():.3e} eV/A (max |F| {np.abs(F_ref).max():.3f})")
    assert err.max() <= F_MAX, (case, precision, float(err.max()))
    # the system evaluates normally afterwards (stored dE/dG and sums rebuilt)
    E, F2 = s.energy_forces()
    E_ref, F2_ref = oracle.energy_forces(c.species, c.coords, c.cell, OW) if c.n <= 2000 else (None, None)
    if E_ref is not None:
        tol = 1e-6 if precision == "fp32" else 1e-3
        assert abs(E - E_ref) <= tol * abs(E_ref)
    s.close()

"""The FP32 brute-force kernel (nb_direct_f32, the paper's bare O(N^2) sum of
Eq. (gravity), Sec. "A Bare Many-body Performance on RV770 GPU") against the
oracle's FP64 direct sum.

The kernel works on positions rounded to FP32, so the oracle sums in FP64 over
exactly those rounded positions: the comparison then isolates the kernel's
arithmetic.  Bars (derived as for the tree's force kernel): a rounded sum's
error scales with A_i = sum_j |a_ij|, about sqrt(k) u A_i for k terms in one
partial sum (u = 6e-8) plus the MUFU rsqrt error (~2^-22 per term).  The tree
path's 1e-5 bar covers lists of ~10^3 terms; a brute-force partial sum holds
up to n/2 terms, so the FP32 bar is 1e-5 x max(1, sqrt(n / 4096)).  The
compensated mode folds each 256-source tile with Kahan's method: 1e-6.
"""
import numpy as np
import pytest

import nbsynth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _run(pos, mass, eps, precision):
    import paper_0909_0541_gb300 as nb
    dev = torch.device("cuda")
    p = torch.from_numpy(np.ascontiguousarray(pos, np.float64)).to(dev)
    m = torch.from_numpy(np.ascontiguousarray(mass, np.float32)).to(dev)
    acc, pot = nb.direct_f32(p, m, eps, precision)
    torch.cuda.synchronize()
    return acc.cpu().numpy().astype(np.float64), pot.cpu().numpy().astype(np.float64)


def _oracle32(pos, mass, eps, targets=None):
    import oracle
    p32 = np.asarray(pos, np.float64).astype(np.float32).astype(np.float64)
    return oracle.direct(p32, mass, eps, targets, with_amag=True)


def _tol(n, precision):
    return 1e-5 * max(1.0, np.sqrt(n / 4096.0)) if precision == "fp32" else 1e-6


CASES = [
    ("plummer", 1, 1.0 / 64), ("plummer", 2, 1.0 / 64), ("plummer", 33, 1.0 / 64),
    ("plummer", 4097, 1.0 / 64), ("cube", 20000, 1e-3), ("halo", 20000, 5e-4),
]


def _set(kind, n):
    if kind == "plummer":
        return nbsynth.plummer(n, 40 + n)
    if kind == "cube":
        return nbsynth.uniform_cube(n, 41 + n)
    return nbsynth.halo_mix(n, 42 + n, n_halos=20)


@pytest.mark.parametrize("precision", ["fp32", "fp32_comp"])
@pytest.mark.parametrize("kind,n,eps", CASES)
def test_direct_f32_matches_oracle(kind, n, eps, precision):
    ps = _set(kind, n)
    acc, pot = _run(ps.pos, ps.mass, eps, precision)
    ra, rp, am = _oracle32(ps.pos, ps.mass, eps)
    tol = _tol(n, precision)
    da = np.linalg.norm(acc - ra, axis=1)
    assert np.all(da <= tol * am + 1e-30), (float(np.max(da / np.maximum(am, 1e-300))), tol)
    # the potential's terms share one sign: relative to |phi|
    if n > 1:
        assert np.all(np.abs(pot - rp) <= tol * np.abs(rp)), \
            float(np.max(np.abs(pot - rp) / np.abs(rp)))
    else:
        assert np.array_equal(acc, np.zeros((1, 3))) and pot[0] == 0.0


def test_direct_f32_two_body_closed_form():
    """Two bodies: |a| = m r / (r^2 + eps^2)^{3/2}, phi = -m / sqrt(r^2 + eps^2)."""
    ps = nbsynth.two_body(0.75, m1=0.25, m2=0.75)
    eps = 0.1
    acc, pot = _run(ps.pos, ps.mass, eps, "fp32")
    r = np.linalg.norm(ps.pos[1] - ps.pos[0])
    s = (r * r + eps * eps) ** 0.5
    m = ps.mass.astype(np.float64)
    assert np.isclose(np.linalg.norm(acc[0]), m[1] * r / s ** 3, rtol=3e-6)
    assert np.isclose(np.linalg.norm(acc[1]), m[0] * r / s ** 3, rtol=3e-6)
    assert np.isclose(pot[0], -m[1] / s, rtol=3e-6)
    assert np.isclose(pot[1], -m[0] / s, rtol=3e-6)


def test_direct_f32_coincident_pairs_contribute_nothing_at_eps0():
    """eps = 0 and coincident particles: such a pair adds nothing (no NaN)."""
    ps = nbsynth.uniform_cube(3000, 77)
    pos = ps.pos.copy()
    pos[1000:1010] = pos[5]                  # eleven particles at one point
    acc, pot = _run(pos, ps.mass, 0.0, "fp32_comp")
    assert np.all(np.isfinite(acc)) and np.all(np.isfinite(pot))
    ra, rp, am = _oracle32(pos, ps.mass, 0.0)
    da = np.linalg.norm(acc - ra, axis=1)
    assert np.all(da <= 1e-6 * am + 1e-30)


def test_direct_f32_sampled_at_1e5():
    """At the crossover sweep's largest size (the launch it times), sampled
    targets against the oracle one by one."""
    ps = nbsynth.uniform_sphere(100_000, 43)
    eps = 1.0 / 64
    acc, pot = _run(ps.pos, ps.mass, eps, "fp32")
    tg = np.random.default_rng(3).choice(ps.n, 512, replace=False)
    ra, rp, am = _oracle32(ps.pos, ps.mass, eps, tg)
    da = np.linalg.norm(acc[tg] - ra, axis=1)
    assert np.all(da <= _tol(ps.n, "fp32") * am)
    assert np.all(np.abs(pot[tg] - rp) <= _tol(ps.n, "fp32") * np.abs(rp))


def test_direct_f32_net_force_vanishes():
    """sum_i m_i a_i = 0 (Newton's third law) to FP32 rounding of the sums."""
    ps = nbsynth.plummer(8192, 44)
    acc, _ = _run(ps.pos, ps.mass, 1.0 / 64, "fp32_comp")
    _, _, am = _oracle32(ps.pos, ps.mass, 1.0 / 64)
    net = (ps.mass[:, None].astype(np.float64) * acc).sum(0)
    assert np.linalg.norm(net) <= 1e-6 * float((ps.mass * am).sum())


def test_direct_f32_rejects_fp64acc_and_small_workspace():
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.plummer(1000, 45)
    dev = torch.device("cuda")
    p = torch.from_numpy(ps.pos).to(dev)
    m = torch.from_numpy(ps.mass).to(dev)
    with pytest.raises(nb.NBError) as ei:
        nb.direct_f32(p, m, 0.01, "fp64acc")
    assert ei.value.code == -1
    small = torch.empty(16, dtype=torch.uint8, device=dev)
    with pytest.raises(nb.NBError) as ei:
        nb.direct_f32(p, m, 0.01, "fp32", work=small)
    assert ei.value.code == -1

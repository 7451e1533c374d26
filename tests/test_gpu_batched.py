"""The batched form: independent instances of uneven size and rank solved by
concurrent workers must give, instance by instance, bitwise the result of a
single solve (the same kernels and fixed-order reductions run), and an
invalid instance must fail alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2311_16019_gb300 import inputs as I  # noqa: E402
from oracle import spkms as SP, measure as M  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_16019_gb300 import build, spk
    build.build()
    return spk.load()


def _opts(P, maxit=120):
    npad = 1 << (P.n1 - 1).bit_length()
    s = min(npad, 2 * P.r * maxit)
    return dict(k=4, s=s, maxit=min(maxit, s // P.r - 1), p=10, tol=1e-8, seed=11,
                precision="fp64")


def test_batched_equals_single_solves_bitwise():
    from paper_2311_16019_gb300 import spk
    probs = I.batched_instances(count=7, seed=9, nmin=12, nmax=40)
    opts = [_opts(P) for P in probs]
    rc, outs = spk.solve_batched(probs, concurrency=3, opts_list=opts, raise_on_error=False)
    assert rc == 0
    for P, o, g in zip(probs, opts, outs):
        single = spk.solve(P.A, P.BT, P.C1, P.C2, raise_on_error=False, **o)
        assert g.X1 is not None and g.iters == single.iters and g.rank == single.rank
        assert torch.equal(g.X1, single.X1) and torch.equal(g.X2, single.X2)


def test_batched_against_oracle_fixed_d():
    """s = 6 (d+1) r keeps the projected spectra in the right half plane for
    these instances (s = 2 d r does not for one of them: see the next test)."""
    from paper_2311_16019_gb300 import spk
    probs = I.batched_instances(count=4, seed=10, nmin=12, nmax=24)
    opts = []
    for P in probs:
        npad = 1 << (P.n1 - 1).bit_length()
        opts.append(dict(_opts(P, maxit=12), s=min(npad, 6 * P.r * 13), fixed_d=12, tol=0.0))
    rc, outs = spk.solve_batched(probs, concurrency=4, opts_list=opts)
    assert rc == 0
    for P, o, g in zip(probs, opts, outs):
        ref = SP.spkms(P.A, P.BT, P.C1, P.C2, k=4, s=o["s"], tol=0.0, maxit=12, p=12, seed=11)
        err = M.rel_error(g.X1.cpu().numpy(), g.X2.cpu().numpy(), ref["X1"], ref["X2"])
        assert err < 1e-10, (P.name, err)


def test_batched_invalid_instance_fails_alone():
    from paper_2311_16019_gb300 import spk
    probs = I.batched_instances(count=3, seed=9, nmin=12, nmax=20)
    opts = [_opts(P) for P in probs]
    opts[1] = dict(opts[1], s=4)          # s < (maxit + 1) r: invalid
    rc, outs = spk.solve_batched(probs, concurrency=2, opts_list=opts, raise_on_error=False)
    assert rc == spk.SPK_ERR_ARG
    assert outs[1].X1 is None and outs[1].status == spk.SPK_ERR_ARG
    assert outs[0].X1 is not None and outs[2].X1 is not None


def test_projected_spectrum_off_right_half_plane_parity():
    """With s = 2 d r this instance's sketched projection has an eigenvalue
    with negative real part (the oracle's H~ has min Re = -41.6, G~'s
    smallest real part is 78: no shift of Eq. (3.4) puts both in the right
    half plane).  The spectral split solves it as the oracle's
    Bartels-Stewart does: X within 1e-10."""
    from paper_2311_16019_gb300 import spk
    from oracle import spkms as SP, measure as M
    P = I.batched_instances(count=4, seed=10, nmin=12, nmax=24)[2]
    kw = dict(k=4, s=48, maxit=12, p=12, tol=0.0, seed=11)
    g = spk.solve(P.A, P.BT, P.C1, P.C2, fixed_d=12, **kw)
    o = SP.spkms(P.A, P.BT, P.C1, P.C2, **kw)
    assert np.linalg.eigvals(o["Ht"]).real.min() < 0
    err = M.rel_error(g.X1.cpu().numpy(), g.X2.cpu().numpy(), o["X1"], o["X2"])
    assert err < 1e-10, err
    assert g.rho == pytest.approx(o["rho"], rel=1e-8)


def test_spectrum_crossing_before_convergence_converges_as_oracle():
    """Instance 38 of the 64-instance batch (n = 112^2, r = 1, s = 4000):
    from d = 294 on one eigenvalue of H~ lies far in the left half plane
    (-1.03e3 at d = 300) before the estimate reaches 1e-8.  Checking every
    20 iterations, the oracle (Bartels-Stewart) converges at d = 300; the
    device solve must too, with the true residual at tol.  The basis is
    numerically degenerate at that d (the spurious eigenvalue is its mark),
    so the projected solution is ill-conditioned: both X solve the equation
    to the same residual and agree to 1e-6, not 1e-10."""
    from paper_2311_16019_gb300 import spk
    from oracle import spkms as SP, measure as M
    P = I.batched_instances(count=64, seed=4)[38]
    kw = dict(k=4, s=4000, maxit=2000, p=20, tol=1e-8, seed=4)
    g = spk.solve(P.A, P.BT, P.C1, P.C2, **kw)
    o = SP.spkms(P.A, P.BT, P.C1, P.C2, **kw)
    assert o["converged"] and g.converged and g.iters == o["d"] == 300
    err = M.rel_error(g.X1.cpu().numpy(), g.X2.cpu().numpy(), o["X1"], o["X2"])
    tres = M.true_residual(P.A, P.B, P.C1, P.C2, g.X1.cpu().numpy(), g.X2.cpu().numpy())
    ores = M.true_residual(P.A, P.B, P.C1, P.C2, o["X1"], o["X2"])
    print(f"instance 38: d={g.iters}, X vs oracle {err:.2e}, true residual {tres:.2e} "
          f"(oracle {ores:.2e})")
    assert err < 1e-6 and tres < 2e-8 and ores < 2e-8


def test_autotuned_concurrency_is_a_candidate_and_results_do_not_depend_on_it():
    from paper_2311_16019_gb300 import spk
    probs = I.batched_instances(count=6, seed=12, nmin=12, nmax=30)
    opts = [_opts(P, maxit=60) for P in probs]
    c = spk.autotune_concurrency(probs, candidates=(1, 3, 6), probe_iters=10, opts_list=opts)
    assert c in (1, 3, 6)
    _, a = spk.solve_batched(probs, concurrency=c, opts_list=opts, raise_on_error=False)
    _, b = spk.solve_batched(probs, concurrency=1, opts_list=opts, raise_on_error=False)
    for x, y in zip(a, b):
        assert x.status == y.status and x.iters == y.iters
        if x.X1 is not None:
            assert torch.equal(x.X1, y.X1) and torch.equal(x.X2, y.X2)

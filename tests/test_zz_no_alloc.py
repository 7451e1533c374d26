"""The allocation-free sketch entry point (spk_sketch_apply_static), for
callers that cannot let the library allocate device memory, against the
handle-based spk_sketch_apply: same output (the tolerance of the sketch
parity tests, and in fact bit-identical: the same kernels run) on two calls
in a row with different sizes, and a clear error beyond the static limits.
Collected last so that a failure here never hides another test's result."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2311_16019_gb300 import build, spk
    build.build()
    return spk.load()


def test_static_scratch_matches_allocating_entry_point_twice():
    from paper_2311_16019_gb300 import spk
    cases = [(3000, 3, 500, 4, 1), (70000, 4, 2000, 9, 0)]
    for n, r, s, seed, sid in cases:
        X = np.random.default_rng(n + r).standard_normal((n, r))
        want = spk.sketch_apply(X, s, seed=seed, sketch_id=sid).cpu().numpy()
        got = spk.sketch_apply_static(X, s, seed=seed, sketch_id=sid).cpu().numpy()
        assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)
        assert np.array_equal(got, want)


def test_static_scratch_rejects_oversize():
    from paper_2311_16019_gb300 import spk
    X = torch.zeros((300000, 4), dtype=torch.float64, device="cuda")  # n' r = 2^21
    with pytest.raises(spk.SpkError) as e:
        spk.sketch_apply_static(X, 100, seed=0, sketch_id=0)
    assert e.value.code == spk.SPK_ERR_ARG and "static scratch" in str(e.value)

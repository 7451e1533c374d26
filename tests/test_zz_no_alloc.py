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


def test_static_scratch_call_allocates_no_device_memory():
    """The property the entry point exists for: after a warm-up call (the
    per-device set-up), a call with other sizes leaves the driver's free
    device memory unchanged.  Input and output are allocated, and the torch
    caching allocator is settled, before the measured call."""
    from paper_2311_16019_gb300 import spk
    lib = spk.load()
    import ctypes as C
    X0 = torch.randn((5000, 2), dtype=torch.float64, device="cuda")
    spk.sketch_apply_static(X0, 300, seed=1, sketch_id=0)          # warm-up / set-up
    X = torch.randn((90000, 4), dtype=torch.float64, device="cuda")
    SX = torch.empty((4, 1500), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    err = C.create_string_buffer(256)
    rc = lib.spk_sketch_apply_static(90000, 1500, 7, 1, C.c_void_p(X.data_ptr()), 4,
                                     C.c_void_p(SX.data_ptr()),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                     err, 256)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert rc == spk.SPK_OK, err.value
    assert free1 == free0
    want = spk.sketch_apply(X, 1500, seed=7, sketch_id=1).cpu().numpy()
    assert np.array_equal(SX.t().cpu().numpy(), want)


def test_static_scratch_rejects_oversize():
    from paper_2311_16019_gb300 import spk
    X = torch.zeros((300000, 4), dtype=torch.float64, device="cuda")  # n' r = 2^21
    with pytest.raises(spk.SpkError) as e:
        spk.sketch_apply_static(X, 100, seed=0, sketch_id=0)
    assert e.value.code == spk.SPK_ERR_ARG and "static scratch" in str(e.value)

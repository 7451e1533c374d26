"""The C-ABI library builds, loads and exports every symbol include/spk.h
declares; its structs match the binding's layout (no GPU compute)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spk.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2311_16019_gb300 import build, spk
    build.build()
    return spk.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spk_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layout_matches_binding(lib):
    from paper_2311_16019_gb300 import spk
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "spk.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(spk_csr), sizeof(spk_opts),
         sizeof(spk_result), offsetof(spk_opts, tol), offsetof(spk_result, X1_dev),
         offsetof(spk_result, ms_recover), sizeof(spk_problem), offsetof(spk_problem, opts),
         offsetof(spk_opts, verify), offsetof(spk_opts, fp64_until),
         offsetof(spk_result, true_rel_res), offsetof(spk_result, switch_d));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    want = [ctypes.sizeof(spk.Csr), ctypes.sizeof(spk.Opts), ctypes.sizeof(spk.Result),
            spk.Opts.tol.offset, spk.Result.X1_dev.offset, spk.Result.ms_recover.offset,
            ctypes.sizeof(spk.Problem), spk.Problem.opts.offset, spk.Opts.verify.offset,
            spk.Opts.fp64_until.offset, spk.Result.true_rel_res.offset,
            spk.Result.switch_d.offset]
    assert got == want


def test_host_only_entry_points(lib):
    from paper_2311_16019_gb300 import spk
    o = spk.Opts()
    lib.spk_opts_default(ctypes.byref(o))
    assert o.k_left == 2 and o.tol == 1e-8 and o.max_newton > 0
    assert lib.spk_status_string(spk.SPK_ERR_NOT_CONVERGED).decode().startswith("not converged")
    assert lib.spk_version() >= 100


def test_create_without_gpu_reports_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    h = ctypes.c_void_p()
    assert lib.spk_create(ctypes.byref(h), 0) == -2  # SPK_ERR_CUDA, no abort
    assert not h.value


def test_product_path_has_no_cpu_fallback():
    """The binding raises when no GPU is visible instead of computing on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_2311_16019_gb300 import inputs as I, spk
    P = I.workload("lap16_r1")
    with pytest.raises(RuntimeError):
        spk.solve(P.A, P.BT, P.C1, P.C2, k=2, s=64, maxit=10)


def test_package_does_not_import_oracle():
    for dirpath, _, files in os.walk(os.path.join(ROOT, "paper_2311_16019_gb300")):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, flags=re.M), f
                assert "oracle/" not in txt, f


def test_plain_c_program_links_and_calls_the_library(lib):
    """A C99 program (no C++, no torch) includes spk.h, links libspk.so and
    calls it: the host-only schedule function and spk_create, which without a
    GPU must return SPK_ERR_CUDA instead of aborting."""
    import torch
    from paper_2311_16019_gb300 import spk
    src = r'''
#include <stdio.h>
#include "spk.h"
int main(void) {
  const int32_t d[3] = {20, 40, 80};
  const double rel[3] = {1e-2, 1e-3, 1e-4};
  int32_t next = spk_next_check(d, rel, 3, 1e-8, 20, 1500);
  spk_handle* h = NULL;
  int rc = spk_create(&h, 0);
  if (rc == SPK_OK) spk_destroy(h);
  printf("%d %d %d\n", (int)next, rc, h == NULL);
  return 0;
}
'''
    libdir = os.path.dirname(spk.LIB_PATH)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I",
                               os.path.join(ROOT, "include"), c, "-o", exe,
                               "-L", libdir, "-lspk", "-Wl,-rpath," + libdir])
        nxt, rc, null = (int(x) for x in subprocess.check_output([exe]).split())
    # the line through (40, -3) and (80, -4) in (d, log10 rel) reaches -8
    # 160 iterations after 80; 80 + ceil(0.7 * 1.05 * 160) = 198 -> 200 (p = 20)
    assert nxt == 200
    if not torch.cuda.is_available():
        assert rc == -2 and null == 1


def test_binding_constants_match_header_enums():
    """The binding's status codes and option values are the header's enums
    (compiled from spk.h, not parsed), so a renumbering on either side fails
    here instead of selecting the wrong sketch, precision or method."""
    from paper_2311_16019_gb300 import spk
    names = ["SPK_OK", "SPK_ERR_ARG", "SPK_ERR_CUDA", "SPK_ERR_ALLOC", "SPK_ERR_BREAKDOWN",
             "SPK_ERR_SINGULAR_PROJECTED", "SPK_ERR_NONFINITE", "SPK_ERR_NOT_CONVERGED",
             "SPK_ERR_TIMEOUT", "SPK_ERR_UNSUPPORTED"]
    enums = {"SPK_SKETCH_SRHT": spk.SKETCH["srht"], "SPK_SKETCH_IDENTITY": spk.SKETCH["identity"],
             "SPK_SKETCH_DCT": spk.SKETCH["dct"], "SPK_PREC_FP64": spk.PRECISION["fp64"],
             "SPK_PREC_MIXED_FP32": spk.PRECISION["mixed_fp32"],
             "SPK_PREC_MIXED_BF16": spk.PRECISION["mixed_bf16"],
             "SPK_CHECK_EVERY_P": spk.CHECK["every_p"], "SPK_CHECK_ADAPTIVE": spk.CHECK["adaptive"],
             "SPK_METHOD_SKETCHED": spk.METHOD["sketched"],
             "SPK_METHOD_TRUNCATED": spk.METHOD["truncated"], "SPK_METHOD_FULL": spk.METHOD["full"],
             "SPK_INJECT_NAN_C1": spk.INJECT_NAN_C1,
             "SPK_INJECT_RANK_DEFICIENT": spk.INJECT_RANK_DEFICIENT,
             "SPK_INJECT_TIMEOUT": spk.INJECT_TIMEOUT, "SPK_INJECT_SINGULAR": spk.INJECT_SINGULAR}
    enums.update({n: getattr(spk, n) for n in names})
    keys = sorted(enums)
    body = "".join(f'  printf("%ld\\n", (long){k});\n' for k in keys)
    src = '#include <stdio.h>\n#include "spk.h"\nint main(void) {\n' + body + "  return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "e.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "e")
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    assert dict(zip(keys, got)) == {k: enums[k] for k in keys}

"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/msrsb.h declares (no device work)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "msrsb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(msrsb_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_abi():
    names = _declared()
    for want in ("msrsb_filter", "msrsb_build_basis", "msrsb_coarse_op", "msrsb_setup", "msrsb_apply",
                 "msrsb_solve", "msrsb_destroy", "msrsb_partition"):
        assert want in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_06934_gb300 import msrsb as B
    lib = ctypes.CDLL(B.lib_path())
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(B.EXPORTS) == set(_declared())


def test_partition_size_host_only():
    # msrsb_partition_size does no device work, so it runs without a GPU
    from paper_1912_06934_gb300 import msrsb as B
    assert B.msrsb_partition_size(B.grid((64, 64, 64), (8, 8, 8))) == (262144, 512, 8)
    assert B.msrsb_partition_size(B.grid((49, 49, 49), (6, 6, 6), centering=1, ncomp=3)) == (117649, 729, 8)
    assert B.msrsb_partition_size(B.grid((64, 64), (8, 8))) == (4096, 64, 4)


def test_tune_calls_are_host_only():
    # the autotuner's mode and table are host bookkeeping: callable without a GPU
    from paper_1912_06934_gb300 import msrsb as B
    # the binding's struct mirrors the header's field for field
    hdr = open(os.path.join(ROOT, "include", "msrsb.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} msrsb_tune_entry;", hdr).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(int32_t|float)\s+(\w+)(\[\d+\])?;", body)
    assert [f[1] for f in fields] == [f[0] for f in B.c_tune_entry._fields_]
    assert ctypes.sizeof(B.c_tune_entry) == sum(4 * (int(f[2][1:-1]) if f[2] else 1) for f in fields)
    B.msrsb_tune_reset()
    assert B.msrsb_tune_table() == []
    for mode in (B.MSRSB_TUNE_AUTO, 0, 5):
        B.msrsb_tune_mode(mode)
    for bad in (-2, 6, 1000):
        try:
            B.msrsb_tune_mode(bad)
        except B.MsrsbError as e:
            assert e.status == 1  # MSRSB_EINVAL
        else:
            raise AssertionError("mode %d accepted" % bad)
    B.msrsb_tune_mode(B.MSRSB_TUNE_AUTO)
    lib = B.load()
    cnt = ctypes.c_int32(-1)
    assert lib.msrsb_tune_table(None, ctypes.c_int32(-1), ctypes.byref(cnt)) == 1  # negative capacity
    assert lib.msrsb_tune_table(None, ctypes.c_int32(4), ctypes.byref(cnt)) == 1   # no array for 4 entries
    assert lib.msrsb_tune_table(None, ctypes.c_int32(0), ctypes.byref(cnt)) == 0 and cnt.value == 0


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_1912_06934_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_wait_selftest_rejects_bad_limits_on_the_host():
    # the limit is checked before any device work, so this runs without a GPU
    import __graft_entry__
    __graft_entry__.build()
    from paper_1912_06934_gb300 import msrsb as B
    lib = B.load()
    lib.msrsb_wait_selftest.argtypes = [ctypes.c_double, ctypes.c_void_p]
    for lim in (0.0, -1.0, 1000.5, float("nan")):
        assert lib.msrsb_wait_selftest(lim, None) == B.MSRSB_EINVAL


def test_binding_constants_match_the_header():
    # every enumerator of include/msrsb.h has the same value in the binding
    from paper_1912_06934_gb300 import msrsb as B
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "msrsb.h")).read(), flags=re.S)
    found = dict((k, int(v)) for k, v in re.findall(r"\b(MSRSB_[A-Z0-9_]+)\s*=\s*(\d+)", src))
    assert len(found) >= 18
    for name, value in found.items():
        assert getattr(B, name) == value, name


_ALLOC = re.compile(r"\b(cudaMalloc\w*|cudaFree\w*|cudaHostAlloc|cudaMallocHost|dalloc|dfree|malloc|calloc|realloc|"
                    r"free|new|cub)\b")


def _strip_comments(src):
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return re.sub(r'"(?:\\.|[^"\\])*"', '""', src)


def test_noalloc_entry_point_names_no_allocation_call():
    """msrsb_build_basis_noalloc is for callers that cannot allocate device
    memory: its translation unit, and the argument check it calls from another
    one, name no allocation or free routine of CUDA, CUB, C or C++."""
    csrc = os.path.join(ROOT, "paper_1912_06934_gb300", "csrc")
    code = _strip_comments(open(os.path.join(csrc, "noalloc.cu")).read())
    assert not _ALLOC.findall(code)
    # the only function of another translation unit it calls
    calls = set(re.findall(r"\b([a-z_]+)\s*\(", code)) - set(re.findall(r"\b([a-z_]+)\s*\([^;{]*\)\s*\{", code))
    assert "check_mat" in calls
    filt = _strip_comments(open(os.path.join(csrc, "filter.cu")).read())
    body = re.search(r"msrsb_status check_mat\(const msrsb_mat \*A\) \{(.*?)\n\}", filt, flags=re.S).group(1)
    assert not _ALLOC.findall(body)

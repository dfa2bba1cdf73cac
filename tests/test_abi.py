"""C ABI: the library builds, loads without a GPU and exports every function
include/ldlt_rpm.h declares; host-side argument checks return their codes."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libs():
    import __graft_entry__ as g
    g.build()
    import paper_1802_10453_gb300 as lr
    return lr


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|size_t)\s+\**(\w+)\s*\(", txt, flags=re.M)))


def test_exports_match_header(libs):
    names = _declared("ldlt_rpm.h")
    assert "ldlt_rpm_factor" in names and "rpm_from_factor" in names
    out = subprocess.run(["nm", "-D", "--defined-only", libs.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    for nme in names:
        assert nme in exported, nme
    L = libs.lib()
    for nme in names:
        assert hasattr(L, nme)


def test_version(libs):
    assert libs.lib().ldlt_rpm_version() >= 10000


@pytest.mark.parametrize("p,path,code", [
    (65521, 1, 0), (65521, 0, 0), (2147483647, 1, 0), (2, 1, 0), (2, 0, 0),
    (65520, 1, -2), (1, 1, -2), (0, 0, -2), (2147483648 + 11, 1, -3),
    (2147483647, 0, -3), (67108859, 0, 0), (65521, 7, -1),
])
def test_workspace_query_codes(libs, p, path, code):
    out = ctypes.c_size_t(0)
    rc = libs.lib().ldlt_rpm_workspace_bytes(1000, p & 0xFFFFFFFF, path, ctypes.byref(out))
    assert rc == code
    if code == 0:
        assert out.value > 3 * 1000 * 1000 * 4


def test_factor_argument_errors(libs):
    L = libs.lib()
    # composite p, p too large, negative n, bad path: all rejected before any device call
    assert L.ldlt_rpm_factor(4, 15, None, 4, None, None, None, None, 1, None, 0, None) == -2
    assert L.ldlt_rpm_factor(4, 2147483659, None, 4, None, None, None, None, 1, None, 0, None) == -3
    assert L.ldlt_rpm_factor(-1, 7, None, 4, None, None, None, None, 1, None, 0, None) == -1
    assert L.ldlt_rpm_factor(4, 7, None, 4, None, None, None, None, 9, None, 0, None) == -1
    buf = ctypes.create_string_buffer(8)
    # NULL A with n > 0, lda < n
    assert L.ldlt_rpm_factor(4, 7, None, 4, buf, buf, buf, buf, 1, None, 0, None) == -1
    assert L.ldlt_rpm_factor(4, 7, buf, 3, buf, buf, buf, buf, 1, None, 0, None) == -1
    # workspace too small
    assert L.ldlt_rpm_factor(4, 7, buf, 4, buf, buf, buf, buf, 1, buf, 8, None) == -4
    assert L.rpm_from_factor(-1, None, None, None, None, None) == -1


def test_test_drop_codes(libs):
    """The failure-detection hook accepts only its documented codes (host only)."""
    L = libs.lib()
    assert L.ldlt_rpm_test_drop(3) == -1
    assert L.ldlt_rpm_test_drop(-1) == -1
    assert L.ldlt_rpm_test_drop(0) == 0


def test_speculation_default_matches_header(libs):
    hdr = open(os.path.join(ROOT, "include", "ldlt_rpm.h")).read()
    assert int(re.search(r"#define LDLT_SPECULATION_DEFAULT\s+(\d+)", hdr).group(1)) == libs.SPECULATION_DEFAULT
    L = libs.lib()
    assert L.ldlt_rpm_set_speculation(0) == -1 and L.ldlt_rpm_set_speculation(17) == -1
    assert L.ldlt_rpm_set_speculation(libs.SPECULATION_DEFAULT) == 0


def test_effective_ops_formula(libs):
    # Section 6: r^3/3 + n^2 r - r^2 n; r = n gives n^3/3
    assert libs.effective_ops(300, 300) == pytest.approx(300 ** 3 / 3)
    assert libs.effective_ops(16384, 8192) == pytest.approx(7 * 16384 ** 3 / 24)


def test_noalloc_limits_on_host(libs):
    """ldlt_rpm_factor_noalloc refuses what its fixed scratch array cannot hold
    before touching the device, and that array holds every problem up to the
    stated maximum order on both paths."""
    hdr = open(os.path.join(ROOT, "include", "ldlt_rpm.h")).read()
    assert int(re.search(r"#define LDLT_NOALLOC_MAX_N\s+(\d+)", hdr).group(1)) == libs.NOALLOC_MAX_N
    mb = int(re.search(r"#define LDLT_NOALLOC_BYTES\s+\(\(size_t\)(\d+) << 20\)", hdr).group(1))
    assert mb << 20 == libs.NOALLOC_BYTES
    assert int(re.search(r"#define LDLT_ERR_TOO_LARGE\s+(-\d+)", hdr).group(1)) == libs.LDLT_ERR_TOO_LARGE
    assert int(re.search(r"#define LDLT_ERR_INTERNAL\s+(-\d+)", hdr).group(1)) == libs.LDLT_ERR_INTERNAL
    for p in (2, 3, 251, 65521, 8388593, 67108859, 2147483647):
        for path in (libs.PATH_FP64, libs.PATH_TC):
            try:
                need = libs.workspace_bytes(libs.NOALLOC_MAX_N, p, path)
            except libs.LdltError:
                continue
            assert need <= libs.NOALLOC_BYTES, (p, path, need)
    L = libs.lib()
    buf = ctypes.create_string_buffer(8)
    big = libs.NOALLOC_MAX_N + 1
    assert L.ldlt_rpm_factor_noalloc(big, 65521, buf, big, buf, buf, buf, buf, 1, None) == -8
    assert L.ldlt_rpm_factor_noalloc(4, 15, buf, 4, buf, buf, buf, buf, 1, None) == -2
    assert L.ldlt_rpm_factor_noalloc(-1, 7, buf, 4, buf, buf, buf, buf, 1, None) == -1
    assert L.ldlt_rpm_factor_noalloc(4, 7, buf, 4, buf, buf, buf, buf, 5, None) == -1


def test_batched_host_checks(libs):
    """ldlt_rpm_factor_batched rejects bad arguments before any device work."""
    L = libs.lib()
    buf = ctypes.create_string_buffer(1024)
    args = lambda count, p, path, ws, nbytes: (count, buf, p, buf, buf, buf, buf, buf, buf, path, ws, nbytes, None)
    assert L.ldlt_rpm_factor_batched(*args(-1, 7, 1, buf, 1024)) == -1
    assert L.ldlt_rpm_factor_batched(*args(3, 15, 1, buf, 1024)) == -2
    assert L.ldlt_rpm_factor_batched(*args(3, 2147483659, 1, buf, 1024)) == -3
    assert L.ldlt_rpm_factor_batched(*args(3, 7, 9, buf, 1024)) == -1
    assert L.ldlt_rpm_factor_batched(*args(0, 7, 1, None, 0)) == 0          # nothing to do
    assert L.ldlt_rpm_factor_batched(*args(3, 7, 1, None, 0)) == -4
    assert L.ldlt_rpm_factor_batched(*args(3, 7, 1, buf, 1024)) == -4      # less than one CTA's scratch
    assert L.ldlt_rpm_factor_batched(3, None, 7, buf, buf, buf, buf, buf, buf, 1, buf, 1024, None) == -1
    one = 512 * 512 * 4
    assert libs.batched_workspace_bytes(1, 65521) == 256 + 256 + one
    assert libs.batched_workspace_bytes(4096, 65521) == 256 + 4096 * 4 + 640 * one
    with pytest.raises(libs.LdltError):
        libs.batched_workspace_bytes(5, 65520)
    for bad in [(8, 0, 8), (32, -1, 32), (32, 514, 32), (32, 0, 3), (16, 0, 32)]:
        assert L.ldlt_rpm_batched_set_schedule(*bad) == -1
    assert L.ldlt_rpm_batched_set_schedule(32, 0, 32) == 0


def test_strict_host_checks(libs):
    L = libs.lib()
    buf = ctypes.create_string_buffer(64)
    assert L.ldlt_rpm_strict(4, 15, buf, 4, buf, buf, None) == -2
    assert L.ldlt_rpm_strict(-1, 2, buf, 4, buf, buf, None) == -1
    assert L.ldlt_rpm_strict(4, 2, buf, 3, buf, buf, None) == -1
    assert L.ldlt_rpm_strict(4, 2, None, 4, buf, buf, None) == -1
    assert L.ldlt_rpm_strict(4, 7, buf, 4, buf, buf, None) == 0   # odd p: nothing to do, no device work
    assert L.ldlt_rpm_strict(0, 2, None, 1, None, None, None) == 0


def test_solve_host_checks(libs):
    L = libs.lib()
    buf = ctypes.create_string_buffer(256)
    args = lambda n, p, lda, ldb, nrhs, ldx, ws, nb: (n, p, buf, lda, buf, buf, buf, buf, ldb, nrhs, buf, ldx, buf, ws, nb, None)
    assert L.ldlt_rpm_solve(*args(4, 15, 4, 1, 1, 1, buf, 256)) == -2
    assert L.ldlt_rpm_solve(*args(-1, 7, 4, 1, 1, 1, buf, 256)) == -1
    assert L.ldlt_rpm_solve(4, 7, buf, 4, buf, buf, buf, buf, 1, 1, buf, 1, None, buf, 256, None) == -1  # status NULL

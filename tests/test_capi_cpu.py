"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every entry point include/*.h declares, and rejects bad arguments
before touching the device."""
import glob
import os
import re
import subprocess
import sys

import pytest

from paper_2602_21242_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_create_ex", "lbm_init", "lbm_step", "lbm_moments",
                     "lbm_diagnostics", "lbm_get_state", "lbm_set_state", "lbm_destroy", "lbm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = capi.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(lbm_\w+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported


def test_build_targets_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_layout():
    pitch, plane, nbytes = capi.lbm_layout(4096, 4096, capi.LBM_F64)
    assert pitch == 4096 and plane == 4096 * 4096 and nbytes == 9 * 4096 * 4096 * 8
    pitch, plane, nbytes = capi.lbm_layout(33, 7, capi.LBM_F64)
    assert pitch == 48 and (pitch * 8) % 128 == 0 and (plane * 8) % 256 == 0 and plane >= pitch * 7
    pitch, plane, nbytes = capi.lbm_layout(33, 7, capi.LBM_F16_SHIFT)
    assert pitch == 64 and nbytes == 9 * plane * 2
    with pytest.raises(capi.LBMError):
        capi.lbm_layout(0, 5, capi.LBM_F64)
    with pytest.raises(capi.LBMError):
        capi.lbm_layout(5, 5, 7)


@pytest.mark.parametrize("args,fragment", [
    ((0, 8, 1 / 3, 0.6, 3), "invalid size"),
    ((8, 8, 1.2, 0.6, 3), "theta"),
    ((8, 8, 0.0, 0.6, 3), "theta"),
    ((8, 8, 1 / 3, 0.5, 3), "tau"),
    ((8, 8, 1 / 3, float("nan"), 3), "tau"),
    ((8, 8, 1 / 3, 0.6, 6), "model"),
    ((8, 8, 1 / 3, 0.6, -1), "model"),
])
def test_create_rejects_bad_arguments(args, fragment):
    with pytest.raises(capi.LBMError) as e:
        capi.lbm_create(*args)
    assert e.value.status == capi.LBM_EINVAL
    assert fragment in str(e.value)


def test_calls_reject_null_context():
    lib = capi.load()
    assert lib.lbm_step(None, 1) == capi.LBM_EINVAL
    assert lib.lbm_init(None, None, None, None) == capi.LBM_EINVAL
    assert lib.lbm_destroy(None) == capi.LBM_OK
    assert isinstance(capi.last_error(None), str)
    assert capi.lbm_version() >> 16 == 1


# Addresses that are never dereferenced: lbm_step_noalloc checks sizes, ranges and
# overlaps on the host and returns before its first CUDA call when one fails.
_FAR = 1 << 40


@pytest.mark.parametrize("args,fragment", [
    ((0, 8, 1 / 3, 0.6, 3, _FAR, 2 * _FAR, 3 * _FAR), "invalid size"),
    ((8, 8, 1.0, 0.6, 3, _FAR, 2 * _FAR, 3 * _FAR), "out of range"),
    ((8, 8, 1 / 3, 0.5, 3, _FAR, 2 * _FAR, 3 * _FAR), "out of range"),
    ((8, 8, 1 / 3, 0.6, 6, _FAR, 2 * _FAR, 3 * _FAR), "out of range"),
    ((8, 8, 1 / 3, 0.6, 3, 0, 2 * _FAR, 3 * _FAR), "NULL"),
    ((8, 8, 1 / 3, 0.6, 3, _FAR, 0, 3 * _FAR), "NULL"),
    ((8, 8, 1 / 3, 0.6, 3, _FAR, 2 * _FAR, 0), "NULL"),
    # 16384 x 16384 needs 16384 blocks at 64 rows per thread: beyond the fixed scratch
    ((16384, 16384, 1 / 3, 0.6, 3, _FAR, 2 * _FAR, 3 * _FAR), "more than the 8192"),
    # d_dst starts inside d_src, d_diag5 inside d_src, d_diag5 inside d_dst
    ((64, 64, 1 / 3, 0.6, 3, _FAR, _FAR + 8, 3 * _FAR), "overlap"),
    ((64, 64, 1 / 3, 0.6, 3, _FAR, 2 * _FAR, _FAR + 4096), "overlap"),
    ((64, 64, 1 / 3, 0.6, 3, _FAR, 2 * _FAR, 2 * _FAR - 8), "overlap"),
])
def test_noalloc_rejects_bad_arguments_before_touching_the_device(args, fragment):
    with pytest.raises(capi.LBMError) as e:
        capi.lbm_step_noalloc(*args)
    assert e.value.status == capi.LBM_EINVAL
    assert fragment in str(e.value)


def test_product_sources_never_reach_the_oracle():
    """The package, its CUDA sources and the public header name nothing under oracle/:
    no import, include, path or library of the checker."""
    pattern = re.compile(r"\bimport\s+oracle|from\s+oracle\b|liboracle|olbm_oracle|olbm_core|oracle/")
    hits, scanned = [], 0
    for sub in ("paper_2602_21242_gb300", "include"):
        for path in glob.glob(os.path.join(ROOT, sub, "**", "*"), recursive=True):
            if "_build" in path or not path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                continue
            scanned += 1
            for n, line in enumerate(open(path, encoding="utf-8"), 1):
                if pattern.search(line):
                    hits.append(f"{os.path.relpath(path, ROOT)}:{n}: {line.strip()}")
    assert scanned > 20 and not hits, hits


def test_missing_library_fails_loudly(tmp_path):
    """Without liblbm.so (and no way to build it) the binding raises: there is no fallback."""
    code = f"""
import sys
sys.path.insert(0, {ROOT!r})
from paper_2602_21242_gb300 import build, capi
build.LIB = {str(tmp_path / "absent" / "liblbm.so")!r}
def no_build(*a, **k):
    raise RuntimeError("nvcc not found")
build.build = no_build
try:
    capi.load()
except RuntimeError as e:
    print("raised:", e)
    sys.exit(0)
sys.exit(3)
"""
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0 and "raised:" in res.stdout, res.stdout + res.stderr


def test_lattice_without_a_gpu_raises():
    """On a host without CUDA the torch wrapper raises instead of computing anywhere else."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2602_21242_gb300.lattice import Lattice

    with pytest.raises(Exception):
        Lattice(8, 8, 1 / 3, 0.6, "complete")


def test_every_declaration_cites_its_passage():
    """Each function include/*.h declares sits under a comment that names the passage of the
    paper it implements (an equation, section or figure) or says it has no counterpart there."""
    cite = re.compile(r"Eqs?\. \d|Sec\. \d|Fig\. \d|no counterpart in the paper")
    missing = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        comments = [(m.start(), m.end(), re.sub(r"\s*\n\s*\*?\s*", " ", m.group(0)))
                    for m in re.finditer(r"/\*.*?\*/", text, flags=re.S)]
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, flags=re.M):
            if any(a <= m.start(1) < b for a, b, _ in comments):
                continue  # a name inside a comment
            before = [c for a, b, c in comments if b <= m.start()]
            if not before or not cite.search(before[-1]):
                missing.append(m.group(1))
    assert not missing, missing


@pytest.mark.parametrize("args,fragment", [
    (([16, 0], [16, 16], [0.3, 0.3], [0.6, 0.6], 3, capi.LBM_F32_SHIFT), "domain 1: invalid size"),
    (([16], [16], [1.0], [0.6], 3, capi.LBM_F32_SHIFT), "domain 0: theta"),
    (([16, 8], [16, 8], [0.3, 0.3], [0.6, 0.5], 3, capi.LBM_F64), "domain 1: theta"),
    (([16], [16], [0.3], [0.6], 7, capi.LBM_F32_SHIFT), "unknown model"),
    (([16], [16], [0.3], [0.6], 3, capi.LBM_F64_DF), "not available for batches"),
    (([], [], [], [], 3, capi.LBM_F32_SHIFT), "bad arguments"),
])
def test_batch_create_rejects_bad_arguments(args, fragment):
    """lbm_batch_create checks every domain on the host before touching the device."""
    with pytest.raises(capi.LBMError) as e:
        capi.lbm_batch_create(*args)
    assert e.value.status == capi.LBM_EINVAL
    assert fragment in str(e.value)

"""The C-ABI library builds, loads without a GPU, exports every function that
include/*.h declares, and its structs have the layout the Python binding
assumes (checked against a C compiler's sizeof/offsetof)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(relcp_[A-Za-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2506_14097_gb300 import build

    path = build.build()
    return ctypes.CDLL(path), path


def test_exports_every_declared_symbol(lib):
    L, path = lib
    names = declared_functions()
    assert len(names) >= 16
    for nm in sorted(names):
        assert hasattr(L, nm), f"{nm} declared in include/ but not exported by {path}"
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert names <= exported


def test_binding_lists_every_symbol():
    from paper_2506_14097_gb300 import relcp

    assert declared_functions() == set(relcp.EXPORTS)


def test_struct_layout_matches_binding(tmp_path):
    from paper_2506_14097_gb300 import relcp

    prog = tmp_path / "layout.c"
    prog.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "relcp.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(relcp_config), offsetof(relcp_config, dt), offsetof(relcp_config, seed),
         offsetof(relcp_config, flags));
  printf("%zu %zu %zu %zu\\n", sizeof(relcp_step_stats), offsetof(relcp_step_stats, lcp_iters),
         offsetof(relcp_step_stats, lcp_residual), offsetof(relcp_step_stats, steps_done));
  printf("%zu %zu\\n", sizeof(relcp_lcp_info), offsetof(relcp_lcp_info, residual));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    vals = [list(map(int, l.split())) for l in subprocess.check_output([str(exe)], text=True).splitlines()]
    C, S, I = relcp.relcp_config, relcp.relcp_step_stats, relcp.relcp_lcp_info
    assert vals[0] == [ctypes.sizeof(C), C.dt.offset, C.seed.offset, C.flags.offset]
    assert vals[1] == [ctypes.sizeof(S), S.lcp_iters.offset, S.lcp_residual.offset, S.steps_done.offset]
    assert vals[2] == [ctypes.sizeof(I), I.residual.offset]


def test_product_path_does_not_import_oracle():
    """No module of the package imports, loads or executes anything under
    oracle/ (the oracle is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2506_14097_gb300")
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|liboracle|import_module\(\s*['\"]oracle", re.M)
    for f in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            assert not pat.search(open(f).read()), f


def test_enum_constants_match_binding():
    """Every RELCP_* enumerator of include/relcp.h has the same value in the
    Python binding (a flag or status added to one side only fails here)."""
    from paper_2506_14097_gb300 import relcp as R

    src = open(os.path.join(ROOT, "include", "relcp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    found = 0
    for name, val in re.findall(r"\b(RELCP_[A-Z0-9_]+)\s*=\s*(\d+)u?\b", src):
        if hasattr(R, name):
            assert getattr(R, name) == int(val), name
            found += 1
    assert found >= 25
    assert R.RELCP_FLAG_NO_LCP_REFINE == 256


def test_default_lcp_stops():
    """make_config's LCP stop in units of the length scale: 1e-12 on the FP64
    path; on the mixed path 1e-8 for the overdamped laws (the contact velocity
    is the whole non-affine motion of a compaction) and 1e-7 under inertia; an
    explicit lcp_tol is kept."""
    from paper_2506_14097_gb300 import relcp as R

    a = 0.4
    cases = [(R.RELCP_FP64, R.RELCP_OVERDAMPED, 1e-12), (R.RELCP_FP64, R.RELCP_INERTIAL, 1e-12),
             (R.RELCP_MIXED, R.RELCP_OVERDAMPED, 1e-8), (R.RELCP_MIXED, R.RELCP_OVERDAMPED_2D, 1e-8),
             (R.RELCP_MIXED, R.RELCP_INERTIAL, 1e-7)]
    for prec, dyn, k in cases:
        c = R.make_config(dynamics=dyn, precision=prec, eps_ncp=1e-3 * a, length_scale=a)
        assert abs(c.lcp_tol - k * a) <= 1e-15 * k * a, (prec, dyn, c.lcp_tol)
    c = R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=R.RELCP_MIXED, eps_ncp=1e-3 * a, lcp_tol=3e-9)
    assert c.lcp_tol == 3e-9
    # without a length scale the smallest semi-axis is read off eps_ncp = 1e-3 a_min
    c = R.make_config(dynamics=R.RELCP_OVERDAMPED, precision=R.RELCP_MIXED, eps_ncp=1e-3 * a)
    assert abs(c.lcp_tol - 1e-8 * a) <= 1e-20

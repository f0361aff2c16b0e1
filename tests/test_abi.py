"""C-ABI checks that need no GPU: the library loads, exports every function
include/pdcs.h declares, the ctypes mirrors match the C struct layouts, and
argument validation that happens before any device work reports errors."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_2603_15504_b300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdcs.h")


def _declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(pdcs_\w+)\s*\(", text, re.M)))


def test_library_exports_every_declared_function():
    L = P.lib()
    names = _declared_functions()
    assert "pdcs_setup" in names and "pdcs_solve" in names and "pdcs_free" in names
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(P.EXPORTS)


def test_struct_layouts_match_header():
    structs = {"pdcs_cone": P.PdcsCone, "pdcs_options": P.PdcsOptions,
               "pdcs_result": P.PdcsResult, "pdcs_state": P.PdcsState,
               "pdcs_profile": P.PdcsProfile, "pdcs_mlp_config": P.PdcsMlpConfig,
               "pdcs_instance": P.PdcsInstance}
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "%s"' % HEADER, "int main(void){"]
    for cname, cls in structs.items():
        src.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            src.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    src.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write("\n".join(src))
        subprocess.run(["gcc", "-o", exe, c], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = dict(line.split() for line in out.strip().splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(cls, f).offset, (cname, f)


def test_default_options_follow_the_paper():
    o = P.default_options()
    assert o.rel_tol == 1e-6 and o.abs_tol == 1e-6 and o.time_limit == 1000.0
    assert o.use_preconditioner == 1 and o.method == 0 and o.use_adaptive_restart == 1
    # Sec. 3.2.3 direct-API defaults
    assert o.use_adaptive_step_size_weight == 1 and o.use_duality_gap_restart == 1
    assert o.use_kkt_restart == 0 and o.kkt_restart_freq == 2000 and o.print_freq == 2000
    assert o.overlap_launches == 0
    assert o.eps_primal_infeasible_low_acc == 1e-12 and o.eps_dual_infeasible_low_acc == 1e-12
    assert o.eps_primal_infeasible_high_acc == 1e-16 and o.eps_dual_infeasible_high_acc == 1e-16


def _tiny():
    import numpy as np
    return dict(m=2, n=2, row_ptr=np.array([0, 1, 2], np.int64), col_idx=np.array([0, 1], np.int32),
                val=np.ones(2), h=np.zeros(2), c=np.ones(2), nb=2, lo=np.zeros(2),
                hi=np.ones(2), row_cones=[(1, 2)], col_cones=[])


@pytest.mark.parametrize("patch,msg", [
    (dict(row_cones=[(1, 3)]), "sum to m"),
    (dict(row_cones=[(4, 2)]), "dimension 3"),
    (dict(row_cones=[(9, 2)]), "bad row cone"),
    (dict(col_cones=[(1, 1)]), "sum to n - nb"),
    (dict(nb=3), "nb <= n"),
])
def test_invalid_arguments_rejected_before_device_work(patch, msg):
    p = _tiny()
    p.update(patch)
    with pytest.raises(P.PdcsError, match=msg):
        P.Solver(p)


def test_invalid_option_rejected():
    with pytest.raises(P.PdcsError, match="precision"):
        P.Solver(_tiny(), precision=3)
    with pytest.raises(P.PdcsError, match="kkt_restart_freq"):
        P.Solver(_tiny(), use_kkt_restart=1, kkt_restart_freq=0)
    with pytest.raises(P.PdcsError, match="thresholds"):
        P.Solver(_tiny(), eps_dual_infeasible_high_acc=-1.0)


def test_entry_point_build_reaches_the_library_build(monkeypatch):
    """__graft_entry__.build() must call the compiler step of the package (the
    package re-exports a function named build, which shadows the submodule)."""
    import importlib
    import __graft_entry__ as g
    B = importlib.import_module("paper_2603_15504_b300.build")
    calls = []
    monkeypatch.setattr(B, "build", lambda force=False, verbose=False: calls.append((force, verbose)))
    g.build()
    assert calls == [(True, True)]

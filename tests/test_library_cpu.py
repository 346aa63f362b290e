"""CPU checks of the C ABI library: it builds, loads, exports every symbol the
headers declare, and the Python binding's structures match the C layout."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2501_03944_gb300 import build as b
    b.build()
    import paper_2501_03944_gb300 as p
    p.load_library()
    return p


def _declared_symbols():
    names = set()
    for h in ("mgfwa.h", "mgfwa_debug.h"):
        text = open(os.path.join(ROOT, "include", h)).read()
        names |= set(re.findall(r"MGFWA_API\s+[\w\s\*]+?\b(mgfwa_\w+)\s*\(", text))
    return names


def test_exports_every_declared_symbol(pkg):
    declared = _declared_symbols()
    assert declared, "no declarations found"
    assert declared == set(pkg.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mgfwa_\w+)", out))
    assert declared <= exported
    # nothing but the C ABI is exported
    assert exported == declared


def test_structure_layout_matches_header(pkg, tmp_path):
    """Compile a C program against the header and compare every field offset with the ctypes mirror."""
    import ctypes
    classes = (pkg.mgfwa_config, pkg.mgfwa_objective, pkg.mgfwa_info, pkg.mgfwa_request_info,
               pkg.mgfwa_server_stats, pkg.mgfwa_best_key)
    body = []
    for cls in classes:
        body.append(f'  printf("{cls.__name__} %zu\\n", sizeof({cls.__name__}));')
        for fname, _ in cls._fields_:
            body.append(f'  printf("{cls.__name__}.{fname} %zu\\n", offsetof({cls.__name__}, {fname}));')
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"mgfwa.h\"\nint main(void) {\n" +
                   "\n".join(body) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    want = dict(l.rsplit(" ", 1) for l in lines if l)
    for cls in classes:
        assert int(want[cls.__name__]) == ctypes.sizeof(cls), cls.__name__
        for fname, _ in cls._fields_:
            assert int(want[f"{cls.__name__}.{fname}"]) == getattr(cls, fname).offset, (cls.__name__, fname)


def test_config_defaults(pkg):
    cfg = pkg.mgfwa_config_init()
    assert abs(cfg.sigma - 0.2) < 1e-7 and cfg.boost == 1.0
    assert abs(cfg.c_amplify - 1.2) < 1e-7 and abs(cfg.c_reduce - 0.9) < 1e-7
    assert cfg.precision == pkg.MGFWA_FP32


def test_create_rejects_bad_configs_without_a_gpu(pkg):
    """Validation happens before any CUDA call, so EINVAL comes back on a CPU-only host too."""
    import workloads as W
    w = W.MLP_8_16_3
    X, y = W.make_data(w)
    bad = [dict(sparks_per_firework=41), dict(lb=1.0, ub=-1.0), dict(dim=100), dict(eval_budget=2),
           dict(sigma=0.0), dict(precision=7), dict(n_runs=0), dict(loser_out=2), dict(lagged_guiding=-1)]
    for over in bad:
        with pytest.raises(pkg.MgfwaError) as e:
            pkg.Mgfwa.for_workload(w, 0, X=X, y=y, **over)
        assert e.value.status == pkg.MGFWA_EINVAL, over
        assert pkg.mgfwa_last_error() != ""
    ybad = y.copy()
    ybad[3] = 7
    with pytest.raises(pkg.MgfwaError):
        pkg.Mgfwa.for_workload(w, 0, X=X, y=ybad)


def test_network_objective_validation_without_a_gpu(pkg):
    """The testbed network (Sec. 4.1) is checked before any CUDA call: widths from dim to 1, each in
    [1, 4096], at most 16 layers, known activations, parameters given, FP32 only."""
    import workloads as W
    w = W.table2_net(1)
    bad = [dict(precision=pkg.MGFWA_BF16), dict(widths=(10, 16, 2)), dict(widths=(12, 16, 1)),
           dict(widths=(10, 5000, 1), acts=(W.ACT_RELU,)), dict(acts=(W.ACT_RELU, 7, W.ACT_RELU, W.ACT_RELU,
                                                                      W.ACT_RELU, W.ACT_RELU)),
           dict(widths=(10,) + (4,) * 17 + (1,), acts=(W.ACT_RELU,) * 17), dict(params=None),
           dict(refine_every=1, refine_steps=1, refine_lr=0.1)]
    for over in bad:
        kw = dict(dim=w.dim, lb=w.lb, ub=w.ub, n_fireworks=w.n_fireworks, sparks_per_firework=w.sparks_per_firework,
                  guiding_per_firework=w.guiding_per_firework, eval_budget=w.eval_budget, seed=0,
                  kind=pkg.MGFWA_OBJ_NET_OUTPUT, widths=w.widths, acts=w.acts, params=W.make_net(w))
        kw.update(over)
        with pytest.raises(pkg.MgfwaError) as e:
            pkg.Mgfwa(**kw)
        assert e.value.status == pkg.MGFWA_EINVAL, over
    # the MLP objective keeps GELU out
    m = W.MLP_8_16_3
    X, y = W.make_data(m)
    with pytest.raises(pkg.MgfwaError):
        pkg.Mgfwa.for_workload(m, 0, X=X, y=y, acts=(W.ACT_GELU,))


def test_binding_refuses_missing_library(pkg, tmp_path):
    with pytest.raises(ImportError):
        pkg.load_library(str(tmp_path / "nope.so"))

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
    src = tmp_path / "layout.c"
    src.write_text(r"""
#include <stddef.h>
#include <stdio.h>
#include "mgfwa.h"
#define F(T, f) printf("%s.%s %zu\n", #T, #f, offsetof(T, f));
int main(void) {
  printf("mgfwa_config %zu\n", sizeof(mgfwa_config));
  printf("mgfwa_objective %zu\n", sizeof(mgfwa_objective));
  printf("mgfwa_info %zu\n", sizeof(mgfwa_info));
  F(mgfwa_config, dim) F(mgfwa_config, lb) F(mgfwa_config, ub) F(mgfwa_config, n_fireworks)
  F(mgfwa_config, sparks_per_firework) F(mgfwa_config, guiding_per_firework) F(mgfwa_config, sigma)
  F(mgfwa_config, boost) F(mgfwa_config, amp_init) F(mgfwa_config, c_amplify) F(mgfwa_config, c_reduce)
  F(mgfwa_config, eval_budget) F(mgfwa_config, seed) F(mgfwa_config, precision) F(mgfwa_config, elite_rescore)
  F(mgfwa_objective, kind) F(mgfwa_objective, n_layers) F(mgfwa_objective, widths) F(mgfwa_objective, acts)
  F(mgfwa_objective, n_samples) F(mgfwa_objective, X) F(mgfwa_objective, y)
  F(mgfwa_info, evals) F(mgfwa_info, generations) F(mgfwa_info, k) F(mgfwa_info, dim_padded)
  F(mgfwa_info, sparks_per_gen) F(mgfwa_info, device_bytes) F(mgfwa_info, kernel_launches)
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    want = dict(l.rsplit(" ", 1) for l in lines if l)
    for cls in (pkg.mgfwa_config, pkg.mgfwa_objective, pkg.mgfwa_info):
        assert int(want[cls.__name__]) == __import__("ctypes").sizeof(cls), cls.__name__
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
           dict(sigma=0.0), dict(precision=7)]
    for over in bad:
        with pytest.raises(pkg.MgfwaError) as e:
            pkg.Mgfwa.for_workload(w, 0, X=X, y=y, **over)
        assert e.value.status == pkg.MGFWA_EINVAL, over
        assert pkg.mgfwa_last_error() != ""
    ybad = y.copy()
    ybad[3] = 7
    with pytest.raises(pkg.MgfwaError):
        pkg.Mgfwa.for_workload(w, 0, X=X, y=ybad)


def test_binding_refuses_missing_library(pkg, tmp_path):
    with pytest.raises(ImportError):
        pkg.load_library(str(tmp_path / "nope.so"))

"""The bounds-checked debug build against the oracle on small grids.

The library built with -DDIRAC_DEBUG=1 (DIRAC_NVCC_EXTRA, as libdirac_debug.so through
DIRAC_BUILD_TAG=debug) checks the index of every memory access of the line passes against
its buffer; a failed check is recorded in a device flag (no trap) and reported by the next
synchronising call as DIRAC_ECUDA. Every line length of the small grids here runs in that
build, in both precisions, in the default shapes, the persistent pass and the alternative
radix schedules, and must match the oracle with no check failing.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

SCRIPT = r'''
import json, sys
import numpy as np
import oracle
import paper_1909_02894_gb300 as D
from paper_1909_02894_gb300 import workloads as W
oracle.build()
ALT = D.DIRAC_LAUNCH_ALT_RADIX
out = []
for nx, ny in ((16, 16), (32, 16), (16, 64), (128, 32), (256, 16), (16, 512), (1024, 16),
               (2048, 16), (4096, 16)):
    ax, ay = 0.15 * nx, 0.15 * ny
    X, Y = W.mesh(nx, ny, ax, ay)
    g11 = 1.0 + 0.2 * np.exp(-((X - 0.1 * ax) ** 2 + Y ** 2) / (0.2 * ax * ay))
    psi0 = W.wave_packet(nx, ny, ax, ay, 0.1 * min(ax, ay) + 0.5, (1.0, -0.7))
    w = W.Workload("dbg", nx, ny, ax, ay, np.ones((ny, nx)), g11, 1.0 + 0.5 * (g11 - 1.0),
                   mass=0.4, c=1.0, pml_width_x=max(1, nx // 16),
                   pml_width_y=max(1, ny // 16), pml_type=1, sigma0=0.5, theta=0.0,
                   psi0=psi0, dt=0.05, steps=5)
    ref = oracle.run(oracle.Problem.from_workload(w), w.psi0, w.dt, 5)
    for prec in (D.DIRAC_C128, D.DIRAC_C64):
        for shape in (0, 1024, 256 | ALT, 512 | ALT):
            if shape == 1024 and prec == D.DIRAC_C128:
                continue
            with D.Simulation(w, precision=prec) as s:
                D.dirac_set_launch(s.ctx, shape, shape)
                s.set_state(w.psi0)
                s.step(5, w.dt)
                got = s.get_state()
            out.append({"grid": [nx, ny], "prec": prec, "shape": shape,
                        "rel_l2": W.rel_l2(got, ref)})
print(json.dumps(out))
'''


def test_debug_build_matches_the_oracle_with_no_failed_index_check():
    env = dict(os.environ, DIRAC_NVCC_EXTRA="-DDIRAC_DEBUG=1", DIRAC_BUILD_TAG="debug")
    subprocess.run([sys.executable, "-c",
                    "import paper_1909_02894_gb300._build as b; b.build()"],
                   env=env, cwd=ROOT, check=True, timeout=900)
    lib = os.path.join(ROOT, "paper_1909_02894_gb300", "libdirac_debug.so")
    assert os.path.exists(lib)
    env = dict(os.environ, DIRAC_LIB=lib)
    env.pop("DIRAC_NVCC_EXTRA", None)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(res) == 9 * 7
    for x in res:
        tol = 1e-11 if x["prec"] == 1 else 1e-5
        assert x["rel_l2"] <= tol, x

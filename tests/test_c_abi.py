"""The C ABI from a plain C program: tests/c_abi_example.c is compiled with gcc against
include/mpm.h and libmpm_gb300.so, runs two recorded steps and a reverse pass from host
buffers, and must agree with the same run through the Python binding."""
import os
import subprocess

import numpy as np
import pytest

from paper_2412_12089_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_client_matches_python_binding(tmp_path):
    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300.batch import Batch

    lib_dir = os.path.dirname(mpm.LIB_PATH)
    exe = str(tmp_path / "c_abi_example")
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_abi_example.c"), "-L", lib_dir, "-lmpm_gb300",
                           f"-Wl,-rpath,{lib_dir}", "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    c_x, c_xb = (float(t) for t in out.stdout.split())

    # the same environment and inputs through the Python binding
    n = 512
    p = np.arange(n)
    ijk = np.stack([p % 8, (p // 8) % 8, p // 64], 1).astype(np.float32)
    x = (np.float32(0.4) + np.float32(0.025) * (ijk + np.float32(0.5))).astype(np.float32)
    v = np.tile(np.array([0.1, 0.0, -0.05], np.float32), (n, 1))
    spec = wl.EnvSpec(n_particles=n, grid_res=32, substeps=5, dt=1e-4, material="neohookean", E=1e4, nu=0.3,
                      rho=1e3, p_vol=0.008 / n, n_sub=n)
    init = wl.EnvInit(x, v, np.zeros((n, 3, 3), np.float32), np.broadcast_to(np.eye(3, dtype=np.float32),
                                                                             (n, 3, 3)).copy())
    b = Batch([spec], max_steps=2)
    try:
        b.set_inits([init])
        for _ in range(2):
            b.step(None, record=True)
        xf = b.get_state()["x"].cpu().numpy().astype(np.float64)
        g = b.backward(xb=np.ones((n, 3), np.float32))
        xb0 = g["xb0"].cpu().numpy().astype(np.float64)
    finally:
        b.close()
    assert abs(c_x - xf.sum()) <= 1e-6 * abs(xf.sum()), (c_x, xf.sum())
    assert abs(c_xb - xb0.sum()) <= 1e-5 * abs(xb0).sum(), (c_xb, xb0.sum())

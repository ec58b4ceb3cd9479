"""The C-ABI library builds, loads without a GPU and exports every entry point that
include/mpm.h declares; the ctypes structs match the C layout (compiled with gcc)."""
import ctypes as ct
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2412_12089_gb300 import build as b
    from paper_2412_12089_gb300 import mpm

    b.build()
    return mpm.lib()


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpm_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared()
    assert "mpm_create" in names and "mpm_backward" in names and "mpm_submit" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts(tmp_path):
    from paper_2412_12089_gb300 import mpm

    prog = tmp_path / "sizes.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mpm.h"\nint main(){printf("%zu %zu %zu %zu %zu '
                    '%zu %zu\\n", sizeof(mpm_env_spec), sizeof(mpm_options), sizeof(mpm_request), '
                    'sizeof(mpm_result), sizeof(mpm_server_options), offsetof(mpm_env_spec, dt), '
                    'offsetof(mpm_env_spec, pose0));return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ct.sizeof(mpm.MpmEnvSpec), ct.sizeof(mpm.MpmOptions), ct.sizeof(mpm.MpmRequest),
            ct.sizeof(mpm.MpmResult), ct.sizeof(mpm.MpmServerOptions), mpm.MpmEnvSpec.dt.offset,
            mpm.MpmEnvSpec.pose0.offset]
    assert got == want


def test_header_constants_match_binding(tmp_path):
    from paper_2412_12089_gb300 import mpm

    names = ["MPM_STEP_RECORD", "MPM_FLAG_DOMAIN", "MPM_FLAG_NAN", "MPM_FLAG_INVERTED", "MPM_FLAG_WAIT"]
    prog = tmp_path / "consts.c"
    prog.write_text('#include <stdio.h>\n#include "mpm.h"\nint main(){'
                    + "".join(f'printf("%u\\n", (unsigned)({n}));' for n in names) + "return 0;}\n")
    exe = tmp_path / "consts"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == [getattr(mpm, n) for n in names]


def test_invalid_spec_rejected_without_gpu_work(lib):
    """mpm_create validates specs before touching the device."""
    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300 import workloads as wl

    good = wl.cube(n=64).specs[0]
    nan = float("nan")
    cases = [(good.replace(grid_res=30), "grid_res"), (good.replace(grid_res=4), "grid_res"),
             (good.replace(grid_res=132), "grid_res"), (good.replace(n_particles=0), "n_particles"),
             (good.replace(n_particles=1 << 20), "n_particles"), (good.replace(substeps=0), "substeps"),
             (good.replace(dt=0.0), "dt"), (good.replace(dt=nan), "dt"), (good.replace(E=-1.0), "E/nu"),
             (good.replace(nu=0.5), "E/nu"), (good.replace(bound=16), "bound")]
    for spec, word in cases:
        with pytest.raises(mpm.MpmError) as ei:
            mpm.mpm_create([good, spec])
        assert ei.value.code == 1 and "env 1" in str(ei.value) and word in str(ei.value), (word, str(ei.value))
    with pytest.raises(mpm.MpmError) as ei:
        mpm.mpm_create([])
    assert ei.value.code == 1 and "n_envs" in str(ei.value)


def test_invalid_fem_meshes_rejected_without_gpu_work(lib):
    """FEM specs: vertex indices, element groups, collider and mesh size are validated first."""
    import numpy as np

    from paper_2412_12089_gb300 import mpm
    from paper_2412_12089_gb300 import workloads as wl

    good = wl.softjumper(n_envs=1, T=1).specs[0]
    tets = good.fem_tets.copy()
    tets[7, 2] = good.n_particles  # out of range
    grp = good.fem_group.copy()
    grp[3] = good.n_groups
    flat = good.fem_rest.copy()
    flat[good.fem_tets[5]] = flat[good.fem_tets[5][0]]  # element 5 collapses to a point
    cases = [(good.replace(fem_tets=tets), "fem_tets"), (good.replace(fem_group=grp), "fem_group"),
             (good.replace(fem_rest=flat), "degenerate"),
             (good.replace(collider="capsule", act_map=(0,)), "collider"),
             (good.replace(nu=0.0), "nu"),
             (good.replace(n_particles=3000, fem_rest=np.zeros((3000, 3), np.float32)), "n_particles")]
    for spec, word in cases:
        with pytest.raises(mpm.MpmError) as ei:
            mpm.mpm_create([spec])
        assert ei.value.code == 1 and word in str(ei.value), (word, str(ei.value))


def test_product_path_never_imports_oracle():
    """The package sources do not reference the oracle (it is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2412_12089_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "mpm_oracle" not in txt, f

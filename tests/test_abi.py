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


def comment_blocks():
    """Each declared entry point with the comment block that documents it: the comment that
    ends nearest above its declaration, with only other declarations between them (a group of
    declarations shares one block)."""
    src = open(HEADER).read()
    out = {}
    last_comment, last_end = "", -1
    pos = 0
    for m in re.finditer(r"/\*.*?\*/|\b(mpm_[a-z_0-9]+)\s*\(", src, flags=re.S):
        if m.group(0).startswith("/*"):
            gap = src[last_end:m.start()] if last_end >= 0 else ""
            last_comment, last_end = m.group(0), m.end()
            continue
        name = m.group(1)
        # the text between the block and this declaration holds only declarations
        between = src[last_end:m.start()]
        if "#define" in between or "typedef" in between or "enum" in between:
            out.setdefault(name, "")
        else:
            out.setdefault(name, last_comment)
    return out


# The entry points the hot-path boundary names: the batch context, the transition, the
# reverse pass and the request calls.
BOUNDARY = ["mpm_create", "mpm_destroy", "mpm_set_state", "mpm_get_state", "mpm_step", "mpm_backward",
            "mpm_submit", "mpm_poll", "mpm_last_error"]


def test_every_declaration_cites_its_passage():
    """Every entry point's comment block names the paper passage that defines its operation
    (Sec., App., Alg.), or says that the paper has none (systems calls)."""
    blocks = comment_blocks()
    for name in BOUNDARY:
        assert name in blocks, name
    bad = []
    for name, block in blocks.items():
        m = re.search(r"Passage:(.*?)(\*/|\n \*\s*\n|$)", block, flags=re.S)
        if not m:
            bad.append((name, "no Passage line"))
            continue
        text = m.group(1)
        if not (re.search(r"\b(Sec|App|Alg|Eq)\. ?[0-9A-Z]", text) or "none" in text):
            bad.append((name, text.strip()[:60]))
    assert not bad, bad
    for name in ("mpm_step", "mpm_backward", "mpm_create", "mpm_set_state", "mpm_get_state"):
        assert re.search(r"Passage:.*?\b(Sec|App|Alg)\.", blocks[name], flags=re.S), name


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
    for kw, word in ((dict(max_steps=-1), "max_steps"), (dict(max_steps=100001), "max_steps"),
                     (dict(chunk=128), "chunk")):
        with pytest.raises(mpm.MpmError) as ei:
            mpm.mpm_create([good], **kw)
        assert ei.value.code == 1 and word in str(ei.value), (kw, str(ei.value))


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


def test_binning_entry_points_validate_before_device_work(lib):
    """mpm_bin / mpm_bin_static reject bad sizes, grids and pointers before any launch, and
    an empty input is a no-op (all without a GPU)."""
    import numpy as np

    from paper_2412_12089_gb300 import mpm

    x = np.zeros((4, 3), np.float32)
    k = np.zeros(4, np.uint32)
    p = np.zeros(4, np.uint32)
    for fn in (mpm.mpm_bin, mpm.mpm_bin_static):
        for args in ((x, -1, 32, k, p), (x, 4, 30, k, p), (x, 4, 4, k, p), (x, 4, 132, k, p), (None, 4, 32, k, p),
                     (x, 4, 32, None, p), (x, 4, 32, k, None)):
            with pytest.raises(mpm.MpmError) as ei:
                fn(*args)
            assert ei.value.code == 1, (fn.__name__, args[1:3])
        assert fn(x, 0, 32, k, p) == 0
    big = mpm.mpm_bin_static_max() + 1
    with pytest.raises(mpm.MpmError) as ei:
        mpm.mpm_bin_static(x, big, 32, k, p)
    assert ei.value.code == 1


_NULL_CALLS = """
import ctypes as ct
from paper_2412_12089_gb300 import mpm
L = mpm.lib()
N = None
calls = {
    "mpm_set_state": (N,) * 8, "mpm_get_state": (N,) * 7, "mpm_step": (N, N, N, 0, N),
    "mpm_backward": (N,) * 13, "mpm_backward_begin": (N,) * 6, "mpm_backward_step": (N,) * 6,
    "mpm_backward_end": (N,) * 8, "mpm_reset_tape": (N,), "mpm_check_status": (N, N),
    "mpm_time_kernel": (N, 0), "mpm_kernel_time": (N, N, N), "mpm_observe": (N, N, N),
    "mpm_set_obs_adjoint": (N, N, N), "mpm_autotune": (N, 3, N, N), "mpm_autotune_config": (N, N, N, N, N),
    "mpm_submit": (N, N, N), "mpm_poll": (N, 0, N), "mpm_wait": (N, 0, 1.0, N), "mpm_release": (N, 0),
}
bad = {k: getattr(L, k)(*a) for k, a in calls.items()}
L.mpm_destroy(None)
L.mpm_server_destroy(None)
getters = (L.mpm_n_envs(None), L.mpm_n_particles(None), L.mpm_action_dim(None), L.mpm_tape_length(None),
           L.mpm_device_bytes(None), L.mpm_kernel_launches(None), L.mpm_obs_dim(None))
print(repr((bad, getters, L.mpm_last_error(None), L.mpm_server_last_error(None))))
"""


def test_null_handles_are_rejected_not_dereferenced(lib):
    """Every entry point that takes a context or server handle returns INVALID_ARG for a NULL
    one, getters return 0, destroy is a no-op, and the error strings say why; run in a child
    process so that a dereference would show as a crash, not take the test runner down."""
    import ast
    import sys

    out = subprocess.run([sys.executable, "-c", _NULL_CALLS], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    bad, getters, err, serr = ast.literal_eval(out.stdout.strip().splitlines()[-1])
    assert all(code == 1 for code in bad.values()), bad
    assert all(g == 0 for g in getters), getters
    assert b"null" in err and b"null" in serr


def test_server_options_validated_before_device_work(lib):
    from paper_2412_12089_gb300 import mpm

    for kw in (dict(mem_fraction=0.0), dict(mem_fraction=1.5), dict(max_resident=0), dict(chunk=128)):
        with pytest.raises(mpm.MpmError) as ei:
            mpm.mpm_server_create(**kw)
        assert ei.value.code == 1, kw


def test_product_path_never_imports_oracle():
    """The package sources do not reference the oracle (it is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2412_12089_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "mpm_oracle" not in txt, f

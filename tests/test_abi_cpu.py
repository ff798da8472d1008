"""Host-only checks of the C ABI: the library builds, loads without a GPU,
exports every entry point that include/pf.h declares, and the ctypes struct
layouts match the C compiler's.  No CUDA computation is launched."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2302_13612_gb300 import build, pf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return pf.load_library()


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    assert set(names) == set(pf.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pf_\w+)", out))
    assert set(names) <= exported


def test_host_only_entry_points(lib):
    assert lib.pf_strerror(pf.PF_OK) == b"ok"
    assert lib.pf_strerror(pf.PF_ENOCONV).startswith(b"Moulinec")
    c = pf.config_default()
    assert (c.nx, c.ny, c.nz) == (32, 32, 32)
    assert c.C_hex[0] == 59.4 and c.C_hex[4] == 16.4
    assert c.gamma_tw == 0.129 and c.c_over_a == 1.633
    assert abs(c.c2 - 0.03125 * 0.5625) < 1e-15
    assert lib.pf_launch_count(None) == 0
    h = ctypes.c_void_p(123)
    # argument validation happens before any CUDA call
    assert lib.pf_create(None, 1, ctypes.byref(h)) == pf.PF_EINVAL and h.value is None
    bad = pf.config_default()
    bad.nx = 7  # prime factor 7 is not supported
    bad.n_variants = 7
    assert lib.pf_create(ctypes.byref(bad), 1, ctypes.byref(h)) == pf.PF_EINVAL
    dup = pf.config_default()
    dup.n_variants = 2
    dup.variant_ids[0] = dup.variant_ids[1] = 3  # one variant twice
    assert lib.pf_create(ctypes.byref(dup), 1, ctypes.byref(h)) == pf.PF_EINVAL and h.value is None
    assert lib.pf_fma_peak(7, None, None) == pf.PF_EINVAL
    assert lib.pf_step(None, 1, None, None) == pf.PF_EINVAL
    assert lib.pf_energy(None, 0, None) == pf.PF_EINVAL
    assert c.load_mode == pf.PF_LOAD_STRAIN and list(c.load_dir) == [0.0, 0.0, 1.0]
    for mode, d in ((pf.PF_LOAD_UNIAXIAL, (0.0, 0.0, 0.0)), (pf.PF_LOAD_UNIAXIAL, (float("nan"), 0.0, 1.0)),
                    (5, (0.0, 0.0, 1.0))):
        bad = pf.config_default()
        bad.load_mode = mode
        for i in range(3):
            bad.load_dir[i] = d[i]
        assert lib.pf_create(ctypes.byref(bad), 1, ctypes.byref(h)) == pf.PF_EINVAL
    for name, val in (("pic_iters", 65), ("clamp", 2), ("mob_corr", -1)):
        bad = pf.config_default()
        setattr(bad, name, val)
        assert lib.pf_create(ctypes.byref(bad), 1, ctypes.byref(h)) == pf.PF_EINVAL
    assert c.pic_iters == 1 and c.clamp == 0 and c.mob_corr == 3
    bad = pf.config_default()
    bad.warm_degree = 6
    assert lib.pf_create(ctypes.byref(bad), 1, ctypes.byref(h)) == pf.PF_EINVAL
    # least-squares warm start: warm_degree + 1 .. 6 held solutions, degree >= 1
    for deg, pts in ((0, 3), (2, 2), (3, 7), (1, -1)):
        bad = pf.config_default()
        bad.warm_degree, bad.warm_points = deg, pts
        assert lib.pf_create(ctypes.byref(bad), 1, ctypes.byref(h)) == pf.PF_EINVAL, (deg, pts)
    assert c.warm_points == 0
    # anisotropic gradient: all three positive, single crystal only
    for c2, grains in (((0.1, 0.0, 0.2), 1), ((0.1, -0.2, 0.2), 1), ((0.1, 0.2, 0.3), 2)):
        bad = pf.config_default()
        for i in range(3):
            bad.c2_aniso[i] = c2[i]
        bad.n_grains = grains
        R = (ctypes.c_double * 18)(*([1, 0, 0, 0, 1, 0, 0, 0, 1] * 2))
        bad.grain_R = ctypes.cast(R, ctypes.POINTER(ctypes.c_double))
        assert lib.pf_create(ctypes.byref(bad), 1, ctypes.byref(h)) == pf.PF_EINVAL


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stddef.h>
#include <stdio.h>
#include "pf.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(pf_config), offsetof(pf_config, precision),
         offsetof(pf_config, C_hex), offsetof(pf_config, ms_tol), offsetof(pf_config, grain_R),
         offsetof(pf_config, stream), offsetof(pf_config, load_mode), offsetof(pf_config, load_dir),
         offsetof(pf_config, warm_degree), offsetof(pf_config, c2_aniso), offsetof(pf_config, mob_corr),
         offsetof(pf_config, clamp), offsetof(pf_config, autotune), offsetof(pf_config, warm_points),
         sizeof(pf_step_info), offsetof(pf_step_info, mean_strain), offsetof(pf_step_info, mob_change),
         offsetof(pf_step_info, pic_change));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    C = pf.PfConfig
    assert vals == [ctypes.sizeof(C), C.precision.offset, C.C_hex.offset, C.ms_tol.offset,
                    C.grain_R.offset, C.stream.offset, C.load_mode.offset, C.load_dir.offset, C.warm_degree.offset,
                    C.c2_aniso.offset, C.mob_corr.offset, C.clamp.offset, C.autotune.offset,
                    C.warm_points.offset, ctypes.sizeof(pf.PfStepInfo), pf.PfStepInfo.mean_strain.offset,
                    pf.PfStepInfo.mob_change.offset, pf.PfStepInfo.pic_change.offset]

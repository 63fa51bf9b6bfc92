"""C ABI checks that need no GPU: the library loads, exports every entry
point include/pvr.h declares, the Python binding's ctypes structures have
the C layout (checked against a gcc-compiled probe of the header), and the
host-side argument checks reject bad inputs before touching a device."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pvr.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^PVR_API\s+[\w\s\*]+?\b(pvr_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def pvr():
    from paper_1611_07289_b300 import build
    build.build()
    from paper_1611_07289_b300 import pvr as m
    return m


def test_every_declared_symbol_is_exported(pvr):
    names = _declared()
    assert len(names) >= 17
    lib = C.CDLL(pvr.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pvr.exported_symbols())


def test_struct_layout_matches_header(pvr):
    probe = r'''
#include <stddef.h>
#include <stdio.h>
#include "pvr.h"
#define F(T, m) printf(#T "." #m " %zu\n", offsetof(T, m))
int main(void) {
  printf("pvr_geometry %zu\npvr_params %zu\npvr_patches %zu\n", sizeof(pvr_geometry), sizeof(pvr_params), sizeof(pvr_patches));
  F(pvr_geometry, world_to_voxel); F(pvr_geometry, pixel_to_world); F(pvr_geometry, thickness);
  F(pvr_params, psf_dz); F(pvr_params, alpha); F(pvr_params, patch_rule); F(pvr_params, n_params);
  F(pvr_params, reg_grow); F(pvr_params, n_sr); F(pvr_params, max_pixels); F(pvr_params, max_patch_side);
  F(pvr_params, psf_kind); F(pvr_params, psf_sinc_eps); F(pvr_params, slic_a_min);
  F(pvr_params, sr_lambda); F(pvr_params, sr_edge_delta);
  F(pvr_patches, n); F(pvr_patches, max_side); F(pvr_patches, n_pix);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "p.c"), os.path.join(d, "p")
        open(src, "w").write(probe)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(l.split() for l in out if l.strip())
    assert int(got["pvr_geometry"]) == C.sizeof(pvr.Geometry)
    assert int(got["pvr_params"]) == C.sizeof(pvr.Params)
    assert int(got["pvr_patches"]) == C.sizeof(pvr.Patches)
    cls = {"pvr_geometry": pvr.Geometry, "pvr_params": pvr.Params, "pvr_patches": pvr.Patches}
    for k, v in got.items():
        if "." in k:
            t, m = k.split(".")
            assert getattr(cls[t], m).offset == int(v), k


def test_defaults_and_host_argument_checks(pvr):
    p = pvr.default_params()
    assert (p.psf_kxy, p.psf_kz, p.n_params, p.reg_evals) == (1, 3, 6, 40)
    assert abs(p.psf_fwhm_xy - 1.2) < 1e-15 and abs(p.em_c0 - 0.9) < 1e-15
    g = pvr.Geometry()
    g.nx, g.ny, g.nz, g.n_stacks = 1, 8, 8, 1   # nx < 2: rejected on the host
    h = C.c_void_p()
    assert pvr.lib.pvr_ctx_create(C.byref(h), C.byref(g), C.byref(p)) == -1 and not h.value
    g.nx = 8
    g.stack_w[0] = g.stack_h[0] = g.stack_k[0] = 4
    g.pixel_to_world[0][2] = 1.0
    bad = pvr.default_params(psf_kz=99)
    assert pvr.lib.pvr_ctx_create(C.byref(h), C.byref(g), C.byref(bad)) == -1
    bad = pvr.default_params(n_params=7)   # 6 (rigid) and 12 (affine) only
    assert pvr.lib.pvr_ctx_create(C.byref(h), C.byref(g), C.byref(bad)) == -1
    assert pvr.lib.pvr_ctx_create(None, C.byref(g), C.byref(p)) == -1
    # calls on a NULL context fail cleanly
    assert pvr.lib.pvr_simulate(None, None, None, None, None, None, None) == -1
    assert pvr.lib.pvr_last_error(None) == b"null context"


def test_noalloc_host_checks_match_context_creation(pvr):
    """pvr_simulate_noalloc runs the geometry / PSF checks of pvr_ctx_create on
    the host, before any device call: a non-finite matrix, a zero slice axis,
    a bad Taylor-sinc tolerance or an unknown pose size is rejected."""
    def geom():
        g = pvr.Geometry()
        g.nx = g.ny = g.nz = 8
        g.n_stacks = 1
        g.stack_w[0] = g.stack_h[0] = g.stack_k[0] = 4
        for i, v in enumerate((1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0)):
            g.world_to_voxel[i] = v
            g.pixel_to_world[0][i] = v
        g.thickness[0] = 1.0
        return g
    dummy = C.c_void_p(16)   # never dereferenced: the checks fail first
    pt = pvr.Patches(dummy, 1, 4, 16, None)
    p = pvr.default_params()

    def call(g, prm):
        return pvr.lib.pvr_simulate_noalloc(C.byref(g), C.byref(prm), dummy, C.byref(pt), dummy, dummy,
                                            dummy, None)
    g = geom()
    g.pixel_to_world[0][3] = float("nan")
    assert call(g, p) == -1
    g = geom()
    g.world_to_voxel[5] = float("inf")
    assert call(g, p) == -1
    g = geom()
    g.pixel_to_world[0][10] = 0.0   # slice axis (column 2) becomes zero
    assert call(g, p) == -1
    g = geom()
    g.nx = g.ny = g.nz = 2048       # 2^33 voxels
    assert call(g, p) == -1
    assert call(geom(), pvr.default_params(psf_kind=1, psf_sinc_eps=0.0)) == -1
    assert call(geom(), pvr.default_params(n_params=7)) == -1
    assert call(geom(), pvr.default_params(psf_dz=float("nan"))) == -1

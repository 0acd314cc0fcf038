"""The C ABI library: it loads without a GPU, exports every function that
include/cfdem.h declares, and the Python binding's structs have the header's
layout (checked against gcc's offsetof on the header itself)."""
import os
import subprocess
import tempfile

import pytest

from paper_2211_01185_gb300 import cfdem as cf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2211_01185_gb300 import build as B
    B.build()
    return cf.lib()


def test_exports_every_declared_function(lib):
    names = cf.header_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert "sm_103a" in cf.cfdem_version()


def test_struct_layout_matches_header():
    prog = r'''
#include <stddef.h>
#include <stdio.h>
#include "cfdem.h"
#define P(s, f) printf(#s "." #f " %zu\n", offsetof(s, f))
int main(void) {
  printf("cfdem_params %zu\n", sizeof(cfdem_params));
  printf("cfdem_stats %zu\n", sizeof(cfdem_stats));
  P(cfdem_params, rho_f); P(cfdem_params, g); P(cfdem_params, scheme);
  P(cfdem_params, qcm_radius); P(cfdem_params, l2_smoothing); P(cfdem_params, drag_model);
  P(cfdem_params, precision); P(cfdem_params, cg_rtol); P(cfdem_params, cg_maxit);
  P(cfdem_params, eps_floor); P(cfdem_params, pressure_degree); P(cfdem_params, max_radius);
  P(cfdem_params, bin_edge); P(cfdem_params, cg_precond); P(cfdem_params, shear_force); P(cfdem_params, fluid_drag); P(cfdem_params, qcm_conserve);
  P(cfdem_params, autotune);
  P(cfdem_stats, cg_iterations); P(cfdem_stats, cg_relres); P(cfdem_stats, nb);
  P(cfdem_stats, bin_edge); P(cfdem_stats, qcm_radius); P(cfdem_stats, n_pnodes);
  P(cfdem_stats, stage_ms); P(cfdem_stats, kernel_launches); P(cfdem_stats, precond);
  P(cfdem_stats, tile_shape); P(cfdem_stats, tuned); P(cfdem_stats, tune_ms);
  P(cfdem_stats, fdm_tile);
  printf("cfdem_bed_io %zu\n", sizeof(cfdem_bed_io));
  P(cfdem_bed_io, n); P(cfdem_bed_io, x); P(cfdem_bed_io, p_nodal); P(cfdem_bed_io, eps_nodal);
  P(cfdem_bed_io, F_q); P(cfdem_bed_io, host_x); P(cfdem_bed_io, host_p_nodal);
  P(cfdem_bed_io, host_F_elem);
  printf("cfdem_dem_params %zu\n", sizeof(cfdem_dem_params));
  P(cfdem_dem_params, rolling_friction); P(cfdem_dem_params, wall_rolling_friction);
  P(cfdem_dem_params, g); P(cfdem_dem_params, hi); P(cfdem_dem_params, max_radius);
  P(cfdem_dem_params, capacity); P(cfdem_dem_params, precision);
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe], text=True).split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    import ctypes as C
    assert int(got["cfdem_params"]) == C.sizeof(cf.cfdem_params)
    assert int(got["cfdem_stats"]) == C.sizeof(cf.cfdem_stats)
    assert int(got["cfdem_bed_io"]) == C.sizeof(cf.cfdem_bed_io)
    assert int(got["cfdem_dem_params"]) == C.sizeof(cf.cfdem_dem_params)
    for key, val in got.items():
        if "." in key:
            s, f = key.split(".")
            cls = getattr(cf, s)
            assert getattr(cls, f).offset == int(val), key


def test_defaults_and_host_validation(lib):
    p = cf.cfdem_params_default()
    assert p.cg_rtol == 1e-13 and p.cg_maxit == 2000 and p.eps_floor == 0.05
    assert p.rho_f == 1.2 and p.mu_f == 1.8e-5 and tuple(p.g) == (0.0, 0.0, -9.81)
    # NULL handles are rejected on the host, no device touched
    assert lib.cfdem_set_params(None, None) == cf.EINVAL
    assert lib.cfdem_get_stats(None, None) == cf.EINVAL
    assert lib.cfdem_destroy(None) == cf.OK
    assert lib.cfdem_synchronize(None) == cf.EINVAL


def test_static_pcm_rejects_bad_meshes_on_the_host(lib):
    # Every case returns CFDEM_EINVAL from the host-side checks, before any
    # CUDA call; the particle pointers are never dereferenced.
    fake = 0x1000
    good_o, good_e = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    # 2^30 x 2^30 x 16 elements wraps a 64-bit element count to 0
    assert cf.cfdem_pcm_void_fraction_static(good_o, good_e, (1 << 30, 1 << 30, 16), 1, 1,
                                             fake, fake, fake) == cf.EINVAL
    assert cf.cfdem_pcm_void_fraction_static(good_o, good_e, ((1 << 20) + 1, 1, 1), 1, 1,
                                             fake, fake, fake) == cf.EINVAL
    nan = float("nan")
    assert cf.cfdem_pcm_void_fraction_static((nan, 0, 0), good_e, (4, 4, 4), 1, 1,
                                             fake, fake, fake) == cf.EINVAL
    assert cf.cfdem_pcm_void_fraction_static(good_o, (1.0, float("inf"), 1.0), (4, 4, 4), 1, 1,
                                             fake, fake, fake) == cf.EINVAL
    assert cf.cfdem_pcm_void_fraction_static(good_o, good_e, (4, 4, 4), 4, 1,
                                             fake, fake, fake) == cf.EINVAL


def test_mapped_mesh_rejects_bad_meshes_on_the_host(lib):
    # checked before any CUDA call: an index past the nodes, a non-finite
    # coordinate, a bad degree or margin
    import numpy as np
    from paper_2211_01185_gb300 import synth
    mesh = synth.make_cylinder_mesh(0.05, 0.08, 2, 1, 1, 2)
    conn, nodes = mesh["conn"], mesh["nodes"]
    bad = conn.copy()
    bad[0, 0] = nodes.shape[0]
    with pytest.raises(cf.CfdemError):
        cf.MappedMesh(2, bad, nodes)
    nn = nodes.copy()
    nn[3, 1] = np.nan
    with pytest.raises(cf.CfdemError):
        cf.MappedMesh(2, conn, nn)
    with pytest.raises(cf.CfdemError):
        cf.MappedMesh(4, conn, nodes)
    with pytest.raises(cf.CfdemError):
        cf.MappedMesh(2, conn, nodes, margin=-0.5)

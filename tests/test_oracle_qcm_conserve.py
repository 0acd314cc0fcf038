"""Pins of the volume-conserving quadrature-centred void fraction: every
particle's lens volumes scaled by c_i = V_p,i / S_i, S_i the volume the
plain QCM sum deposits on the mesh.

With the scaling the solid volume on the mesh, sum_q w_q |J| (1 - eps_q),
equals sum_i V_p,i to rounding for any placement, particles touching the
walls included (the plain sum loses the parts of the averaging spheres
outside the mesh); S_i recomputed by vectorised brute force over every
Gauss point agrees; and for an interior particle c_i tends to 1 under mesh
refinement at a fixed averaging radius (the convolution of the two sphere
indicators integrates to |B_R| V_p)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2211_01185_gb300 import synth


def _mesh_case(k, n_el=(3, 4, 3), n=60, seed=3):
    c = synth.make_random_case(seed, n_el=n_el, k=k, n=n, extent=(0.03, 0.04, 0.03))
    return c, O.Mesh(c["origin"], c["extent"], c["n_el"], c["k"])


def _solid_volume(m, eps):
    _, w = O.gauss_rule(m.nq)
    w3 = np.einsum("i,j,k->kji", w, w, w).reshape(-1)        # q = qx + nq (qy + nq qz)
    return float(np.sum((1.0 - eps) * w3[None, :]) * np.prod(m.h))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_conserves_particle_volume_with_walls(k):
    c, m = _mesh_case(k)
    R = O.default_qcm_radius(m)
    vp = float(np.sum(4.0 / 3.0 * math.pi * c["r"] ** 3))
    eps_c, _, _ = O.qcm(m, R, c["x"], c["r"], conserve=True)
    eps_p, _, _ = O.qcm(m, R, c["x"], c["r"])
    assert _solid_volume(m, eps_c) == pytest.approx(vp, rel=1e-12)
    # particles touch the walls: the plain sum loses volume there
    assert abs(_solid_volume(m, eps_p) - vp) > 1e-3 * vp


@pytest.mark.parametrize("k", [1, 2])
def test_weights_match_brute_force(k):
    c, m = _mesh_case(k, n=25, seed=8)
    R = O.default_qcm_radius(m)
    cw = O.qcm_weights(m, R, c["x"], c["r"])
    qp = O.quadrature_points(m).reshape(-1, 3)
    _, w = O.gauss_rule(m.nq)
    w3 = np.tile(np.einsum("i,j,k->kji", w, w, w).reshape(-1), m.n_elem) * np.prod(m.h)
    VR = 4.0 / 3.0 * math.pi * R ** 3
    for i in range(c["x"].shape[0]):
        d = np.linalg.norm(qp - c["x"][i], axis=1)
        S = sum(w3[q] * O.lens_volume(R, c["r"][i], d[q]) for q in np.nonzero(d < R + c["r"][i])[0])
        Vp = 4.0 / 3.0 * math.pi * c["r"][i] ** 3
        assert cw[i] == pytest.approx(Vp / (S / VR), rel=1e-12)


def test_interior_weight_tends_to_one_under_refinement():
    R, r = 2.0e-3, 0.8e-3
    x = np.array([[0.0201, 0.0197, 0.0203]])          # far from the walls of a 0.04 m box
    dev = []
    for ne in (8, 16, 32):
        m = O.Mesh((0.0, 0.0, 0.0), (0.04, 0.04, 0.04), (ne, ne, ne), 2)
        dev.append(abs(O.qcm_weights(m, R, x, np.array([r]))[0] - 1.0))
    assert dev[2] < dev[1] < dev[0]
    assert dev[2] < 1e-3

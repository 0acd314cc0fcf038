"""Location on mapped (curved) Q_k hex meshes on the GPU (cfdem_mapped_*)
against the oracle's Newton inversion: element indices bit-exact, reference
coordinates within 1e-12, on subdivided cylinders of every degree with points
inside and outside; a box written as a mapped mesh gives the box location;
and the interpolation of a field linear in x, which an isoparametric map
reproduces exactly, comes back at the particles."""
import numpy as np
import pytest

from _parity import dev, host
from oracle import oracle as O
from paper_2211_01185_gb300 import cfdem as cf
from paper_2211_01185_gb300 import synth

pytestmark = pytest.mark.gpu


def _gpu_locate(mesh, x):
    import torch
    n = x.shape[0]
    elem = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    xi = torch.zeros((n, 3), dtype=torch.float64, device="cuda:0")
    with cf.MappedMesh(mesh["k"], mesh["conn"], mesh["nodes"]) as mm:
        assert mm.locate(n, dev(x), elem, xi) == cf.OK
        torch.cuda.synchronize()
    return host(elem), host(xi)


def _cloud(rng, R, H, n):
    """Points in the cylinder's bounding box (about a fifth of them outside
    the cylinder) plus a few above and below it."""
    x = np.empty((n, 3))
    x[:, :2] = (2 * rng.random((n, 2)) - 1) * R * 1.05
    x[:, 2] = H * (1.1 * rng.random(n) - 0.05)
    return x


@pytest.mark.parametrize("k", [1, 2, 3])
def test_cylinder_location_matches_oracle(k):
    R, H = 0.05, 0.08
    mesh = synth.make_cylinder_mesh(R, H, 4, 3, 5, k)
    rng = np.random.default_rng(20 + k)
    x = _cloud(rng, R, H, 4000)
    e_ref, xi_ref, miss = O.locate_mapped(k, mesh["conn"], mesh["nodes"], x)
    e, xi = _gpu_locate(mesh, x)
    assert 0 < miss < x.shape[0]
    assert np.array_equal(e, e_ref)
    assert np.allclose(xi, xi_ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_box_as_mapped_mesh_matches_box_location(k):
    origin, extent, n_el = (0.01, -0.02, 0.0), (0.03, 0.04, 0.05), (3, 4, 5)
    mesh = synth.make_box_mapped_mesh(origin, extent, n_el, k)
    rng = np.random.default_rng(k)
    h = np.asarray(extent) / np.asarray(n_el)
    cell = rng.integers(0, n_el, size=(2000, 3))
    x = np.asarray(origin) + (cell + 0.02 + 0.96 * rng.random((2000, 3))) * h
    e, xi = _gpu_locate(mesh, x)
    import torch
    with cf.Context(origin, extent, n_el, k) as ctx:
        eb = torch.zeros(x.shape[0], dtype=torch.int32, device="cuda:0")
        xib = torch.zeros((x.shape[0], 3), dtype=torch.float64, device="cuda:0")
        cf.cfdem_locate(ctx.h, x.shape[0], dev(x), eb, xib)
        cf.cfdem_synchronize(ctx.h)
    assert np.array_equal(e, host(eb))
    assert np.allclose(xi, host(xib), rtol=0, atol=1e-12)


@pytest.mark.parametrize("k", [2, 3])
def test_interpolation_reproduces_linear_fields(k):
    import torch
    R, H = 0.05, 0.08
    mesh = synth.make_cylinder_mesh(R, H, 3, 2, 3, k)
    rng = np.random.default_rng(40 + k)
    x = _cloud(rng, R, H, 2000)
    A = rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    field = mesh["nodes"] @ A.T + b
    n = x.shape[0]
    with cf.MappedMesh(k, mesh["conn"], mesh["nodes"]) as mm:
        elem = torch.zeros(n, dtype=torch.int32, device="cuda:0")
        xi = torch.zeros((n, 3), dtype=torch.float64, device="cuda:0")
        out = torch.zeros((n, 3), dtype=torch.float64, device="cuda:0")
        assert mm.locate(n, dev(x), elem, xi) == cf.OK
        assert mm.interpolate(n, elem, xi, 3, dev(field), out) == cf.OK
        torch.cuda.synchronize()
    e = host(elem)
    inside = e >= 0
    assert inside.sum() > n // 2
    want = x @ A.T + b
    assert np.allclose(host(out)[inside], want[inside], rtol=0,
                       atol=1e-11 * np.abs(want).max())
    assert np.all(host(out)[~inside] == 0.0)


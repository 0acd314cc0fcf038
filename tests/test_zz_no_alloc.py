"""The allocation-free particle-centroid void fraction.

cfdem_pcm_void_fraction_static serves callers that may not allocate device
memory (a solver that owns all of it through its own pool, a loop that must
not take the synchronisation a cudaMalloc can cause): its per-element scratch
is a fixed array compiled into the library.
Here it must give what the context-based entry point gives
(cfdem_void_fraction with the particle-centroid scheme), on two calls in a
row -- the second call must clear what the first left in the shared array --
and refuse a mesh larger than that array.  This file is collected last so
that a run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

from _parity import dev, host, rel_err
from oracle import oracle as O
from paper_2211_01185_gb300 import cfdem as cf
from paper_2211_01185_gb300 import synth

pytestmark = pytest.mark.gpu


def _reference(case, x, r):
    import torch
    prm = dict(case["params"], scheme=1)
    E = int(np.prod(case["n_el"]))
    Q = (case["k"] + 1) ** 3
    with cf.Context(case["origin"], case["extent"], case["n_el"], case["k"], prm) as ctx:
        eps = torch.zeros((E, Q), dtype=torch.float64, device="cuda:0")
        cf.cfdem_void_fraction(ctx.h, x.shape[0], x, r, eps)
        cf.cfdem_synchronize(ctx.h)
    return host(eps)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_static_pcm_matches_context_pcm_twice(k):
    import torch
    case = synth.make_random_case(400 + k, n_el=(7, 5, 9), k=k, n=600,
                                  extent=(0.035, 0.025, 0.045))
    other = synth.make_random_case(500 + k, n_el=(7, 5, 9), k=k, n=350,
                                   extent=(0.035, 0.025, 0.045))
    E = int(np.prod(case["n_el"]))
    Q = (k + 1) ** 3
    for c in (case, other):   # two calls in a row, different inputs
        x, r = dev(c["x"]), dev(c["r"])
        out = torch.full((E, Q), -7.0, dtype=torch.float64, device="cuda:0")
        st = cf.cfdem_pcm_void_fraction_static(c["origin"], c["extent"], c["n_el"], k,
                                               c["x"].shape[0], x, r, out)
        assert st == cf.OK
        torch.cuda.synchronize()
        ref = _reference(c, x, r)
        assert rel_err(host(out), ref) <= 1e-10
        # and directly against the FP64 oracle's particle-centroid scheme
        mesh = O.Mesh(c["origin"], c["extent"], c["n_el"], k)
        want, bad = O.pcm(mesh, c["x"], c["r"])
        assert bad == -1                  # every particle lies in the mesh
        assert rel_err(host(out), want) <= 1e-12


def test_static_pcm_refuses_meshes_beyond_its_scratch():
    import torch
    n_el = (128, 128, 33)                      # 540,672 elements > 524,288
    assert int(np.prod(n_el)) > cf.PCM_STATIC_MAX_ELEMS
    x = torch.zeros((1, 3), dtype=torch.float64, device="cuda:0")
    r = torch.ones(1, dtype=torch.float64, device="cuda:0")
    out = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    st = cf.cfdem_pcm_void_fraction_static((0, 0, 0), (1, 1, 1), n_el, 1, 1, x, r, out)
    assert st == cf.EINVAL

"""Shared-memory layout of the FDM slab transform (k_fdm_slab), checked on the
CPU.

The kernel transforms one z-slab in shared memory: the slab X in "slots"
(the two parity halves of an axis, each starting 16-byte aligned), the
y-transformed slab PT (transposed), and the packed diagonal parity blocks of
the x and y transform matrices.  Each product is one call of a register-tile
GEMM whose threads read rows 0..K of their operands (the last row only by a
prefetch) and columns up to the tile grid's edge.  This file restates that
index arithmetic -- the layout functions of csrc/fdm.cu, the threads' tile
origins and the accesses they make -- and checks, over slab sizes and every
register tile the plan may pick:

* every access lies inside the dynamic shared memory the host asks for;
* vector accesses are aligned (64-bit for 2-float, 128-bit for 4-float);
* the two halves of a product write disjoint words;
* the forward and inverse transforms built from these accesses equal the
  plain 1D parity transforms applied along y and then x.

A layout change that breaks one of these (as a host-side size that no
longer matched the kernel's layout once did) fails here, without a GPU."""
import numpy as np
import pytest


def slab_pad(n):
    return ((n + 7) & ~7) + 4


def slab_axis(n):
    ye = (n + 1) // 2
    oe = (ye + 3) & ~3
    return dict(n=n, ye=ye, oe=oe, yo=n // 2, sl=oe + n // 2)


def slot_of(a, p):
    return p if p < a["ye"] else a["oe"] + (p - a["ye"])


def packed_floats(n):
    return (n + 1) * slab_pad((n + 1) // 2)


def layout(nx, ny):
    ax, ay = slab_axis(nx), slab_axis(ny)
    lx, ly = slab_pad(ax["sl"]), slab_pad(ay["sl"])
    X = 0
    PT = X + ay["sl"] * lx
    MX = PT + ax["sl"] * ly
    MY = MX + packed_floats(nx)
    total = MY + packed_floats(ny)
    # the host's size of the dynamic shared memory (floats)
    host = ay["sl"] * lx + ax["sl"] * ly + packed_floats(nx) + packed_floats(ny)
    return dict(ax=ax, ay=ay, lx=lx, ly=ly, lpx=slab_pad(ax["ye"]), lpy=slab_pad(ay["ye"]),
                X=X, PT=PT, MX=MX, MY=MY, total=total, host=host)


def w32(t):
    return (t + 31) & ~31


def threads_for(nx, ny, tr, tc):
    ax, ay = slab_axis(nx), slab_axis(ny)
    cnt = lambda m, n: ((m + tr - 1) // tr) * ((n + tc - 1) // tc)  # noqa: E731
    t1 = w32(cnt(ay["ye"], ax["sl"])) + w32(cnt(ny // 2, ax["sl"]))
    t2 = w32(cnt(ay["sl"], ax["ye"])) + w32(cnt(ay["sl"], nx // 2))
    return max(t1, t2)


def gemm(sm, AT, lda, B, ldb, C, ldc, M, N, K, TR, TC, trans, total):
    """C = A B over the threads' TR x TC tiles; returns the written words."""
    gm, gn = -(-M // TR), -(-N // TC)
    wa, wb = min(TR, 4), min(TC, 4)
    r0 = (np.arange(gm) * TR)[:, None]                 # tile origins
    c0 = (np.arange(gn) * TC)[None, :]
    # alignment of every vector access (rows advance by lda, ldb: multiples of 4)
    assert lda % 4 == 0 and ldb % 4 == 0 and ldc % 4 == 0
    assert np.all((AT + r0) % wa == 0) and np.all((B + c0) % wb == 0)
    # extents: rows 0..K (the last only prefetched), columns to the tile edge
    assert AT >= 0 and B >= 0
    assert AT + K * lda + gm * TR - 1 < total, "A read past the shared memory"
    assert B + K * ldb + gn * TC - 1 < total, "B read past the shared memory"
    A = np.stack([sm[AT + k * lda: AT + k * lda + gm * TR] for k in range(K)])   # [K][gm TR]
    Bm = np.stack([sm[B + k * ldb: B + k * ldb + gn * TC] for k in range(K)])    # [K][gn TC]
    prod = A.T @ Bm                                                                # [gm TR][gn TC]
    written = []
    if trans:   # C[c][r], vector stores of row groups holding a row < M
        for c in range(N):
            for rg in range(0, gm * TR, wa):
                if rg >= M:
                    continue
                idx = C + c * ldc + rg
                assert rg + wa - 1 < -(-M // 4) * 4 or wa == 2, "store past M rounded up to 4"
                assert idx % wa == 0 and idx + wa - 1 < total
                sm[idx: idx + wa] = prod[rg: rg + wa, c]
                written.extend(range(idx, idx + wa))
    else:
        for r in range(M):
            idx = C + r * ldc
            assert idx + N - 1 < total
            sm[idx: idx + N] = prod[r, :N]
            written.extend(range(idx, idx + N))
    return written


def slab(nx, ny, TR, TC, inv, Mx, My, inp):
    L = layout(nx, ny)
    ax, ay, lx, ly, lpx, lpy = L["ax"], L["ay"], L["lx"], L["ly"], L["lpx"], L["lpy"]
    assert L["host"] == L["total"]
    assert L["PT"] % 4 == 0 and L["MX"] % 4 == 0 and L["MY"] % 4 == 0
    assert packed_floats(nx) % 4 == 0 and packed_floats(ny) % 4 == 0   # 16-byte copies
    total = L["total"]
    sm = np.full(total, np.nan)

    def pack(F, a, base, lp):
        sm[base: base + packed_floats(a["n"])] = 0.0
        for k in range(a["ye"]):
            sm[base + k * lp: base + k * lp + a["ye"]] = F[k, : a["ye"]]
        for k in range(a["yo"]):
            sm[base + (a["ye"] + k) * lp: base + (a["ye"] + k) * lp + a["yo"]] = \
                F[a["oe"] + k, a["oe"]: a["oe"] + a["yo"]]

    pack(Mx.T if inv else Mx, ax, L["MX"], lpx)
    pack(My.T if inv else My, ay, L["MY"], lpy)
    X, PT, MX, MY = L["X"], L["PT"], L["MX"], L["MY"]
    for y in range(ny):
        for x in range(nx):
            sm[X + slot_of(ay, y) * lx + slot_of(ax, x)] = inp[y, x]
    yo, xo = ny // 2, nx // 2
    if not inv:   # y butterfly on the rows of X
        for i in range(yo):
            a = sm[X + i * lx: X + i * lx + ax["sl"]].copy()
            j = X + slot_of(ay, ny - 1 - i) * lx
            b = sm[j: j + ax["sl"]].copy()
            sm[X + i * lx: X + i * lx + ax["sl"]] = a + b
            sm[j: j + ax["sl"]] = a - b
    w1 = gemm(sm, MY, lpy, X, lx, PT, ly, ay["ye"], ax["sl"], ay["ye"], TR, TC, True, total)
    w2 = gemm(sm, MY + ay["ye"] * lpy, lpy, X + ay["oe"] * lx, lx, PT + ay["oe"], ly, yo,
              ax["sl"], yo, TR, TC, True, total)
    assert not set(w1) & set(w2) and all(PT <= i < MX for i in w1 + w2)
    if not inv:   # x butterfly on the rows of PT
        for i in range(xo):
            a = sm[PT + i * ly: PT + i * ly + ay["sl"]].copy()
            j = PT + slot_of(ax, nx - 1 - i) * ly
            b = sm[j: j + ay["sl"]].copy()
            sm[PT + i * ly: PT + i * ly + ay["sl"]] = a + b
            sm[j: j + ay["sl"]] = a - b
    else:         # inverse y unfold on the columns of PT
        for r in range(ax["sl"]):
            for i in range(yo):
                p1, p2 = PT + r * ly + i, PT + r * ly + slot_of(ay, ny - 1 - i)
                a, b = sm[p1], sm[p2]
                sm[p1], sm[p2] = a + b, a - b
    w1 = gemm(sm, PT, ly, MX, lpx, X, lx, ay["sl"], ax["ye"], ax["ye"], TR, TC, False, total)
    w2 = gemm(sm, PT + ax["oe"] * ly, ly, MX + ax["ye"] * lpx, lpx, X + ax["oe"], lx, ay["sl"],
              xo, xo, TR, TC, False, total)
    assert not set(w1) & set(w2) and all(X <= i < PT for i in w1 + w2)
    if inv:       # x unfold on the columns of Y
        for r in range(ay["sl"]):
            for i in range(xo):
                p1, p2 = X + r * lx + i, X + r * lx + slot_of(ax, nx - 1 - i)
                a, b = sm[p1], sm[p2]
                sm[p1], sm[p2] = a + b, a - b
    out = np.empty((ny, nx))
    for y in range(ny):
        for x in range(nx):
            out[y, x] = sm[X + slot_of(ay, y) * lx + slot_of(ax, x)]
    return out


def parity_blocks(n, rng):
    """A random transform, block diagonal in the slots of an n-node axis."""
    a = slab_axis(n)
    G = np.zeros((a["sl"], a["sl"]))
    G[: a["ye"], : a["ye"]] = rng.standard_normal((a["ye"], a["ye"]))
    G[a["oe"]: a["oe"] + a["yo"], a["oe"]: a["oe"] + a["yo"]] = \
        rng.standard_normal((a["yo"], a["yo"]))
    return G


def transform_1d(v, n, G, inv):
    """The plain 1D parity transform of a vector of n values."""
    a = slab_axis(n)
    ye, oe, yo = a["ye"], a["oe"], a["yo"]
    if not inv:   # fold, then the two half products with G^T
        s = np.zeros(a["sl"])
        for p in range(n):
            s[slot_of(a, p)] = v[p]
        for i in range(yo):
            u, w = s[i], s[slot_of(a, n - 1 - i)]
            s[i], s[slot_of(a, n - 1 - i)] = u + w, u - w
        y = np.zeros(a["sl"])
        y[:ye] = G[:ye, :ye].T @ s[:ye]
        y[oe: oe + yo] = G[oe: oe + yo, oe: oe + yo].T @ s[oe: oe + yo]
        return np.array([y[slot_of(a, c)] for c in range(n)])
    y = np.zeros(a["sl"])   # inverse: the half products with G, then unfold
    for c in range(n):
        y[slot_of(a, c)] = v[c]
    r = np.zeros(a["sl"])
    r[:ye] = G[:ye, :ye] @ y[:ye]
    r[oe: oe + yo] = G[oe: oe + yo, oe: oe + yo] @ y[oe: oe + yo]
    for i in range(yo):
        u, w = r[i], r[slot_of(a, n - 1 - i)]
        r[i], r[slot_of(a, n - 1 - i)] = u + w, u - w
    return np.array([r[slot_of(a, p)] for p in range(n)])


SIZES = [(2, 2), (3, 3), (2, 5), (5, 5), (7, 9), (9, 7), (4, 6), (17, 10), (13, 13),
         (25, 21), (33, 33), (49, 49), (64, 66)]
TILES = [(4, 4), (4, 8), (8, 4), (8, 8)]


@pytest.mark.parametrize("nx,ny", SIZES)
def test_slab_accesses_and_result(nx, ny):
    rng = np.random.default_rng(1000 * nx + ny)
    Gx, Gy = parity_blocks(nx, rng), parity_blocks(ny, rng)
    inp = rng.standard_normal((ny, nx))
    for TR, TC in TILES:
        if threads_for(nx, ny, TR, TC) > 1024:
            continue
        for inv in (False, True):
            got = slab(nx, ny, TR, TC, inv, Gx, Gy, inp)
            t = np.stack([transform_1d(inp[:, x], ny, Gy, inv) for x in range(nx)], axis=1)
            want = np.stack([transform_1d(t[y, :], nx, Gx, inv) for y in range(ny)], axis=0)
            assert np.allclose(got, want, rtol=1e-12, atol=1e-12), (TR, TC, inv)


@pytest.mark.parametrize("n", [65, 73])
def test_bench_slab_sizes(n):
    """The Q2 32x32x128 and Q3 24x24x96 slabs, with the 4 x 4 tile the plans
    keep (the others are covered at smaller sizes above)."""
    rng = np.random.default_rng(n)
    G = parity_blocks(n, rng)
    inp = rng.standard_normal((n, n))
    for inv in (False, True):
        got = slab(n, n, 4, 4, inv, G, G, inp)
        t = np.stack([transform_1d(inp[:, x], n, G, inv) for x in range(n)], axis=1)
        want = np.stack([transform_1d(t[y, :], n, G, inv) for y in range(n)], axis=0)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
    L = layout(n, n)
    assert L["total"] * 4 <= 220 * 1024    # the slab form's limit: the slab kernel is used

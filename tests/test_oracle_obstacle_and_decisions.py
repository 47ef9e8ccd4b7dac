"""Pins of two parts of the oracle that the reduction to the uniform scheme
(epsilon = 0) and conservation cannot see.

1. The obstacle penalisation of Sec. 7.2.2: after the collision, a leaf C
   takes phi f^eq(rho0, 0) + (1 - phi) f, with phi the share of C inside the
   disc, estimated (reading) by the finest-cell centres of C that lie in the
   closed disc.  The disc is placed so that every quantity is a dyadic
   rational: the centre on a finest-cell centre, the radius three finest
   cells.  Then the count of centres per leaf is a count of integer lattice
   points (a^2 + b^2 <= 9: 29 points in all, Gauss's circle count N(3)), the
   test checks hand-counted values for single leaves, a centre exactly on
   the circle is inside, and the equilibrium at rest comes from the moment
   matrix and equilibria typed from Sec. 7.2.2 in the tests, not from the
   oracle.

2. The detail norm of Def. Details / Eq. Thresholding and the decisions of
   T_eps and H_eps in d = 2 and d = 3.  The test rebuilds, from the leaves
   alone and in numpy: the projection (Def. Projection), the full
   reconstruction below the leaves, the prediction of Sec. 4.1 as the tensor
   product of the one-dimensional operator of Table 1 (the Appendix 2
   construction; a different evaluation order from the oracle's axis and
   diagonal sums), the details of every cell of R(Lambda) and the norm of
   each sibling group (max over the 2^d siblings and over all populations).
   It compares them with the oracle's group norms element by element; then,
   from its own norms, it builds T_eps (with the tree closure), H_eps (the
   neighbour rule k - eta^h and the refinement rule) and the grading
   (every tree cell's parent has its (2s+1)^d neighbourhood in the tree,
   closed by adding only forced cells) from the set definitions, and
   compares the resulting leaves with the oracle's adaptation.
"""
import itertools

import numpy as np
import pytest

from oracle import Oracle
from paper_2103_02903_gb300 import workloads as W
from test_oracle_pins import _ref_scheme


# ---------------------------------------------------------------------------
# 1. obstacle penalisation (Sec. 7.2.2)
# ---------------------------------------------------------------------------

J_OBS = 5          # finest level: [0, 2] x [0, 1] with 2 x 1 roots -> 64 x 32 cells, dx = 1/32
I0, J0 = 11, 11    # the disc is centred on the centre of finest cell (11, 11)
R_CELLS = 3        # radius: three finest cells


def _obstacle_config(obstacle):
    cfg, _ = W.ns_obstacle_2d(seed=1, max_level=J_OBS, min_level=2)
    dx = 1.0 / (1 << J_OBS)
    cfg["phys"][0:6] = [1.0, 0.05, 0.0, (I0 + 0.5) * dx, (J0 + 0.5) * dx, R_CELLS * dx]
    cfg["obstacle"] = obstacle
    return cfg


def _obstacle_mesh():
    """A graded tree: level 3 everywhere, level-3 cells x, y in {2, 3}
    refined to level 4 (finest cells 8..15 on both axes), and level-4 cell
    (5, 5) refined to level 5 (finest cells 10, 11)."""
    leaves = []
    for y in range(8):
        for x in range(16):
            if 2 <= x <= 3 and 2 <= y <= 3:
                for cy in range(2):
                    for cx in range(2):
                        X, Y = 2 * x + cx, 2 * y + cy
                        if (X, Y) == (5, 5):
                            leaves += [(5, 2 * X + a, 2 * Y + b) for b in range(2) for a in range(2)]
                        else:
                            leaves.append((4, X, Y))
            else:
                leaves.append((3, x, y))
    return leaves


def _lattice_count(level, x, y):
    """Finest-cell centres of leaf (level, x, y) in the closed disc, counted
    on the integer lattice: a centre is at offset (a, b) finest cells from
    the disc's centre, inside iff a^2 + b^2 <= R^2."""
    w = 1 << (J_OBS - level)
    n = 0
    for by in range(w):
        for bx in range(w):
            a, b = x * w + bx - I0, y * w + by - J0
            n += a * a + b * b <= R_CELLS * R_CELLS
    return n


def _feq_rest(cfg):
    """Equilibrium populations at (rho0, 0, 0) from the moment matrix and the
    equilibrium moments typed from Sec. 7.2.2."""
    eta, M, Minv, S, meq, cons, m, q = _ref_scheme(cfg)
    mo = np.array([float(v) for v in meq([np.float64(cfg["phys"][0]), np.float64(0.0), np.float64(0.0)])[0]])
    return Minv @ mo


def _collide(cfg, f):
    """One collision of Eq. AdaptiveCollision per column of f (the tests' own
    restatement of Sec. 7.2.2)."""
    eta, M, Minv, S, meq, cons, m, q = _ref_scheme(cfg)
    mo = M @ f
    eq = np.array([np.asarray(v, float) * np.ones(f.shape[1]) for v in meq([mo[0], mo[1], mo[2]])[0]])
    mo = (1 - S[0][:, None]) * mo + S[0][:, None] * eq
    return Minv @ mo


def _obstacle_run(obstacle, collide=True):
    cfg = _obstacle_config(obstacle)
    o = Oracle(cfg)
    leaves = _obstacle_mesh()
    lev = np.array([c[0] for c in leaves], np.int32)
    ix = np.array([c[1] for c in leaves], np.int32)
    iy = np.array([c[2] for c in leaves], np.int32)
    rng = np.random.default_rng(7)
    rho = 1.0 + 0.05 * rng.standard_normal(len(leaves))
    ux = 0.05 + 0.01 * rng.standard_normal(len(leaves))
    uy = 0.01 * rng.standard_normal(len(leaves))
    eta, M, Minv, S, meq, cons, m, q = _ref_scheme(cfg)
    mo = np.array([np.asarray(v, float) * np.ones(len(leaves)) for v in meq([rho, rho * ux, rho * uy])[0]])
    f = Minv @ mo + 1e-3 * rng.standard_normal((9, len(leaves)))  # off equilibrium
    o.set_leaves(lev, ix, iy, np.zeros_like(ix), f)
    o.stream_collide(collide=collide)
    lv, x, y, _, out = o.leaves()
    order = {c: i for i, c in enumerate(zip(lv.tolist(), x.tolist(), y.tolist()))}
    perm = np.array([order[c] for c in leaves])
    return cfg, leaves, out[:, perm]


def test_obstacle_lattice_counts_by_hand():
    """Hand counts of the lattice points a^2 + b^2 <= 9 in single leaves (the
    test's count function, checked before it is used as the expected phi)."""
    assert sum(_lattice_count(*c) for c in _obstacle_mesh()) == 29  # Gauss: N(3) = 29
    assert _lattice_count(5, 10, 10) == 1 and _lattice_count(5, 11, 11) == 1
    assert _lattice_count(4, 5, 4) == 3   # offsets (-1,-3) (0,-3) (-1,-2) (0,-2): 10, 9, 5, 4
    assert _lattice_count(4, 4, 4) == 1   # (-3,-3) (-2,-3) (-3,-2) (-2,-2): 18, 13, 13, 8
    assert _lattice_count(4, 7, 5) == 1   # (3,-1) (4,-1) (3,0) (4,0): 10, 17, 9 on the circle, 16
    assert _lattice_count(4, 6, 5) == 4   # (1,-1) (2,-1) (1,0) (2,0)
    assert _lattice_count(3, 0, 0) == 0


def test_obstacle_penalisation_after_collision():
    cfg, leaves, with_obs = _obstacle_run(1)
    _, _, without = _obstacle_run(0)
    feq = _feq_rest(cfg)
    hit = 0
    for i, (l, x, y) in enumerate(leaves):
        n = _lattice_count(l, x, y)
        w2 = 1 << (2 * (J_OBS - l))
        if n == 0:
            # untouched: the same bits as without the obstacle
            assert np.array_equal(with_obs[:, i], without[:, i]), (l, x, y)
            continue
        hit += 1
        phi = n / w2
        want = phi * feq + (1.0 - phi) * without[:, i]
        np.testing.assert_allclose(with_obs[:, i], want, rtol=1e-14, atol=1e-15, err_msg=str((l, x, y, n)))
        if n == w2:
            # phi = 1: the leaf is the rest equilibrium at rho0
            np.testing.assert_allclose(with_obs[:, i], feq, rtol=1e-14, atol=1e-16)
    # leaves touched: the four level-5 cells and the level-4 leaves around them
    assert hit == 4 + sum(1 for c in leaves if c[0] == 4 and _lattice_count(*c) > 0)
    # the leaf whose only inside centre lies on the circle is penalised
    k = leaves.index((4, 7, 5))
    np.testing.assert_allclose(with_obs[:, k], 0.25 * feq + 0.75 * without[:, k], rtol=1e-14, atol=1e-15)
    assert not np.allclose(with_obs[:, k], without[:, k], rtol=0, atol=1e-9)


def test_obstacle_order_is_distinguishable():
    """Penalising before the collision gives a different result on a
    partially covered leaf, so the previous test does pin the order."""
    cfg, leaves, streamed = _obstacle_run(0, collide=False)
    _, _, with_obs = _obstacle_run(1)
    feq = _feq_rest(cfg)
    k = leaves.index((4, 5, 4))  # phi = 3/4
    phi = 0.75
    before = _collide(cfg, (phi * feq + (1 - phi) * streamed[:, k])[:, None])[:, 0]
    assert np.abs(before - with_obs[:, k]).max() > 1e-8


# ---------------------------------------------------------------------------
# 2. group norms and the T / H decisions in d = 2, 3
# ---------------------------------------------------------------------------

W1 = {0: (0.125, 1.0, -0.125), 1: (-0.125, 1.0, 0.125)}  # Table 1, s = 1: weights of offsets -1, 0, +1


class _Tree:
    """Dense per-level arrays of a tree given by its leaves; coordinates
    (x, y, z), cells per axis n[l][a] = roots_a 2^l."""

    def __init__(self, cfg, d, leaves, f):
        self.cfg, self.d = cfg, d
        self.Jmin, self.J = cfg["min_level"], cfg["max_level"]
        self.per = [cfg["bc"][2 * a] == "periodic" for a in range(d)]
        self.shape = {l: tuple(cfg["roots"][a] << l for a in range(d)) for l in range(self.Jmin, self.J + 1)}
        Q = f.shape[0]
        self.Q = Q
        self.leaf = {l: np.zeros(self.shape[l], bool) for l in self.shape}
        self.F = {l: np.zeros((Q,) + self.shape[l]) for l in self.shape}
        for i, (l, *c) in enumerate(leaves):
            self.leaf[l][tuple(c)] = True
            self.F[l][(slice(None),) + tuple(c)] = f[:, i]
        # R(Lambda): leaves and their ancestors
        self.inR = {l: self.leaf[l].copy() for l in self.shape}
        for l in range(self.J, self.Jmin, -1):
            up = self._coarsen_any(self.inR[l])
            self.inR[l - 1] |= up
        # projection bottom-up on internal cells (Def. Projection)
        for l in range(self.J - 1, self.Jmin - 1, -1):
            internal = self.inR[l] & ~self.leaf[l]
            avg = self._children_mean(self.F[l + 1])
            self.F[l][:, internal] = avg[:, internal]
        # reconstruction top-down below the leaves (Sec. 4.4)
        for l in range(self.Jmin + 1, self.J + 1):
            pred = self.predict(self.F[l - 1])
            self.F[l][:, ~self.inR[l]] = pred[:, ~self.inR[l]]

    def _coarsen_any(self, a):
        out = a
        for ax in range(self.d):
            s = list(out.shape)
            s[ax] //= 2
            s.insert(ax + 1, 2)
            out = out.reshape(s).any(axis=ax + 1)
        return out

    def _children_mean(self, F):
        out = F
        for ax in range(self.d):
            s = list(out.shape)
            s[ax + 1] //= 2
            s.insert(ax + 2, 2)
            out = out.reshape(s).sum(axis=ax + 2)
        return out / (1 << self.d)

    def _shifted(self, A, ax, off):
        """A[.., k + off, ..] along axis ax (of the cell axes), constant
        extension outside a non-periodic domain, wrap on a periodic one."""
        n = A.shape[ax + 1]
        idx = np.arange(n) + off
        idx = idx % n if self.per[ax] else np.clip(idx, 0, n - 1)
        return np.take(A, idx, axis=ax + 1)

    def predict(self, Fc):
        """Values of all cells of the next level predicted from the coarse
        field Fc: the tensor product of the one-dimensional operator."""
        out = Fc
        for ax in range(self.d):
            sh = [self._shifted(out, ax, o) for o in (-1, 0, 1)]
            kids = [W1[c][0] * sh[0] + W1[c][1] * sh[1] + W1[c][2] * sh[2] for c in (0, 1)]
            st = np.stack(kids, axis=ax + 2)  # child parity right after the coarse index
            s = list(out.shape)
            s[ax + 1] *= 2
            out = st.reshape(s)
        return out

    def group_norms(self):
        """G[l][parent] = max over the 2^d children in R and all populations
        of |F - P(F_{l})| (Def. Details), -1 where the parent is not internal."""
        G = {}
        for l in range(self.Jmin, self.J):
            det = np.abs(self.F[l + 1] - self.predict(self.F[l])).max(axis=0)
            det = np.where(self.inR[l + 1], det, -np.inf)
            g = det
            for ax in range(self.d):
                s = list(g.shape)
                s[ax] //= 2
                s.insert(ax + 1, 2)
                g = g.reshape(s).max(axis=ax + 1)
            internal = self.inR[l] & ~self.leaf[l]
            G[l] = np.where(internal, g, -1.0)
        return G


def _close(cells, Jmin, roots_lmin):
    """Add siblings and ancestors (with their siblings) and every level-Jmin cell."""
    out = set(cells)
    for c in itertools.product(*[range(r) for r in roots_lmin]):
        out.add((Jmin,) + c)
    for (l, *k) in list(out):
        k = tuple(k)
        while l > Jmin:
            p = tuple(v // 2 for v in k)
            for off in itertools.product((0, 1), repeat=len(k)):
                out.add((l,) + tuple(2 * pv + o for pv, o in zip(p, off)))
            l, k = l - 1, p
            out.add((l,) + k)
    return out


def _adapt_from_definitions(tr, G, eps, mu_bar, eta, s_pred=1):
    d, Jmin, J = tr.d, tr.Jmin, tr.J
    roots = tr.shape[Jmin]
    epsl = lambda l: eps * 2.0 ** (d * (l - J))
    par = lambda k: tuple(v // 2 for v in k)

    def nbr(l, k):
        out = []
        for a in range(d):
            v, n = k[a], tr.shape[l][a]
            if v < 0 or v >= n:
                if not tr.per[a]:
                    return None
                v %= n
            out.append(v)
        return tuple(out)

    R = {(l,) + tuple(int(v) for v in k) for l in tr.shape for k in zip(*np.nonzero(tr.inR[l]))}
    T = _close({c for c in R if c[0] > Jmin and G[c[0] - 1][par(c[1:])] >= epsl(c[0])}, Jmin, roots)
    H = set(T)
    for c in T:
        l, k = c[0], c[1:]
        for e in eta:
            nb = nbr(l, tuple(k[a] - e[a] for a in range(d)))
            if nb is not None:
                H |= _close({(l,) + nb}, Jmin, roots)
        if Jmin < l < J and G[l - 1][par(k)] >= 2.0 ** (mu_bar + d) * epsl(l):
            kids = {(l + 1,) + tuple(2 * v + o for v, o in zip(k, off)) for off in itertools.product((0, 1), repeat=d)}
            H |= _close(kids, Jmin, roots)
    # grading: add only what Def. Grading forces, until nothing is missing
    tree = set(H)
    changed = True
    while changed:
        changed = False
        for c in list(tree):
            l, k = c[0], c[1:]
            if l == Jmin:
                continue
            p = par(k)
            for off in itertools.product(range(-s_pred, s_pred + 1), repeat=d):
                nb = nbr(l - 1, tuple(p[a] + off[a] for a in range(d)))
                if nb is not None and (l - 1,) + nb not in tree:
                    tree |= _close({(l - 1,) + nb}, Jmin, roots)
                    changed = True
    leaves = set()
    for c in tree:
        l, k = c[0], c[1:]
        if l == J or (l + 1,) + tuple(2 * v for v in k) not in tree:
            leaves.add(c)
    return leaves


def _random_graded_leaves(cfg, d, rng, frac):
    """Leaves of a random graded tree: a random share of the finest cells
    refined down to, then closed under siblings, ancestors and the grading."""
    Jmin, J = cfg["min_level"], cfg["max_level"]
    shapeJ = tuple(cfg["roots"][a] << J for a in range(d))
    per = [cfg["bc"][2 * a] == "periodic" for a in range(d)]
    roots = tuple(cfg["roots"][a] << Jmin for a in range(d))
    seeds = {(J,) + tuple(int(rng.integers(n)) for n in shapeJ) for _ in range(max(1, int(frac * np.prod(shapeJ))))}
    tree = _close(seeds, Jmin, roots)
    changed = True
    while changed:
        changed = False
        for c in list(tree):
            l, k = c[0], c[1:]
            if l == Jmin:
                continue
            for off in itertools.product((-1, 0, 1), repeat=d):
                nb = []
                for a in range(d):
                    v, n = k[a] // 2 + off[a], cfg["roots"][a] << (l - 1)
                    if v < 0 or v >= n:
                        if not per[a]:
                            break
                        v %= n
                    nb.append(v)
                else:
                    if (l - 1,) + tuple(nb) not in tree:
                        tree |= _close({(l - 1,) + tuple(nb)}, Jmin, roots)
                        changed = True
    return sorted(c for c in tree if c[0] == J or (c[0] + 1,) + tuple(2 * v for v in c[1:]) not in tree)


def _case(name, seed, J2=5, J3=4):
    if name == "euler_copy":
        cfg, _ = W.euler_2d(seed=seed, max_level=J2, min_level=2)
        d = 2
    elif name == "d2q9_periodic":
        cfg, _ = W.vortices_2d(seed=seed, max_level=J2, min_level=2)
        d = 2
    else:
        cfg, _ = W.advection_3d(seed=seed, max_level=J3, min_level=2)
        d = 3
    return cfg, d


def _leaf_data(cfg, d, leaves, Q, rng):
    """Smooth fields plus noise of different sizes per population, so that
    the largest detail of a group comes from different populations."""
    J = cfg["max_level"]
    pos = np.array([[(c[1 + a] + 0.5) / (cfg["roots"][a] << c[0]) for a in range(d)] for c in leaves])
    f = np.empty((Q, len(leaves)))
    for p in range(Q):
        k = rng.uniform(1, 6, d)
        ph = rng.uniform(0, 6.3, d)
        base = np.prod(np.sin(2 * np.pi * k * pos + ph), axis=1)
        scale = 10.0 ** rng.uniform(-3, -1)
        f[p] = 1.0 + 0.3 * base + scale * rng.standard_normal(len(leaves))
    return f


def _blob_data(cfg, d, leaves, Q, rng):
    """A constant per population (reproduced exactly by the prediction, with
    the constant extension and with the periodic wrap) plus noise in a small
    ball: details vanish outside the ball, so T coarsens everything else
    down to J_min in one step and the grading has to rebuild the levels in
    between."""
    pos = np.array([[(c[1 + a] + 0.5) / (cfg["roots"][a] << c[0]) for a in range(d)] for c in leaves])
    ball = ((pos - rng.uniform(0.3, 0.7, d)) ** 2).sum(axis=1) < 0.06 ** 2
    f = np.empty((Q, len(leaves)))
    for p in range(Q):
        f[p] = 1.0 + rng.uniform(-0.2, 0.2) + 10.0 ** rng.uniform(-3, -1) * rng.standard_normal(len(leaves)) * ball
    return f


def _to_arrays(leaves, d):
    lev = np.array([c[0] for c in leaves], np.int32)
    xs = [np.array([c[1 + a] for c in leaves], np.int32) for a in range(d)]
    while len(xs) < 3:
        xs.append(np.zeros_like(lev))
    return lev, xs


def _oracle_leaf_set(o, d):
    lev, ix, iy, iz, _ = o.leaves()
    cols = [ix, iy, iz][:d]
    return set(zip(lev.tolist(), *[c.tolist() for c in cols]))


def _check_adaptation(cfg, d, leaves, f, eps_quantile):
    """Group norms against the oracle's, then the adapted leaves against the
    set definitions; returns the test's leaves with and without grading."""
    tr = _Tree(cfg, d, leaves, f)
    G = tr.group_norms()

    # threshold inside the spread of the norms, so that T and H decide both ways
    J = cfg["max_level"]
    scaled = np.concatenate([G[l][G[l] >= 0] / 2.0 ** (d * (l + 1 - J)) for l in G])
    eps = float(np.quantile(scaled[scaled > 1e-10], eps_quantile))
    while True:
        ratios = [abs(g / (eps * 2.0 ** (d * (l + 1 - J)) * t) - 1) for l in G for g in G[l][G[l] >= 0]
                  for t in (1.0, 2.0 ** (cfg["mu_bar"] + d))]
        if min(ratios) > 1e-9:
            break
        eps *= 1.001
    cfg = dict(cfg, eps=eps)

    o = Oracle(cfg)
    lev, xs = _to_arrays(leaves, d)
    o.set_leaves(lev, xs[0], xs[1], xs[2], f)
    assert o.graded()
    o.adapt()
    for l in range(tr.Jmin, tr.J):
        got = o.group_norms(l)
        # the oracle's dense arrays are x fastest: reshape to (z, y, x), then to (x, y, z)
        got = got.reshape(tr.shape[l][::-1]).transpose(tuple(range(d))[::-1])
        want = G[l]
        np.testing.assert_array_equal(got < 0, want < 0, err_msg="internal cells differ at level %d" % l)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14, err_msg="group norms at level %d" % l)

    eta, *_ = _ref_scheme(cfg)
    eta = [tuple(e) + (0,) * (d - len(e)) for e in eta]
    want_leaves = _adapt_from_definitions(tr, G, eps, cfg["mu_bar"], eta)
    got_leaves = _oracle_leaf_set(o, d)
    assert got_leaves == want_leaves
    old_tree = {(l,) + tuple(int(v) for v in k) for l in tr.shape for k in zip(*np.nonzero(tr.inR[l]))}
    ungraded = _adapt_from_definitions(tr, G, eps, cfg["mu_bar"], eta, s_pred=0)
    return got_leaves, old_tree, ungraded


@pytest.mark.parametrize("name", ["euler_copy", "d2q9_periodic", "d3q6_periodic"])
@pytest.mark.parametrize("seed", [0, 1])
def test_group_norms_and_decisions_from_definitions(name, seed):
    """Random graded mesh, noise of mixed sizes everywhere."""
    cfg, d = _case(name, seed)
    rng = np.random.default_rng(1000 + seed)
    leaves = _random_graded_leaves(cfg, d, rng, 0.04 if d == 2 else 0.002)
    assert len({c[0] for c in leaves}) >= 3  # a mesh over several levels
    f = _leaf_data(cfg, d, leaves, W.NPOP[cfg["scheme"]], rng)
    got, old_tree, _ = _check_adaptation(cfg, d, leaves, f, 0.5)
    # the decisions were not trivial: some groups coarsened, some cells refined
    old = set(leaves)
    assert any(c in old_tree and c not in old for c in got)  # an internal cell became a leaf
    assert any((c[0] - 1,) + tuple(v // 2 for v in c[1:]) in old for c in got)  # a leaf was split


@pytest.mark.parametrize("name", ["euler_copy", "d2q9_periodic", "d3q6_periodic"])
@pytest.mark.parametrize("seed", [0, 1])
def test_multilevel_coarsening_and_grading_from_definitions(name, seed):
    """The full finest mesh (as after the initialisation of Algorithm 1) with
    details only in a small ball: coarsening spans several levels at once
    and, for the axis lattices, the grading adds cells the rules of H do not."""
    cfg, d = _case(name, seed, J2=6, J3=5)
    rng = np.random.default_rng(2000 + seed)
    J = cfg["max_level"]
    leaves = [(J,) + c for c in itertools.product(*[range(cfg["roots"][a] << J) for a in range(d)])]
    f = _blob_data(cfg, d, leaves, W.NPOP[cfg["scheme"]], rng)
    got, _, ungraded = _check_adaptation(cfg, d, leaves, f, 0.3)
    levels = {c[0] for c in got}
    assert min(levels) <= J - 3 and J in levels
    if name != "d2q9_periodic":  # the diagonal neighbours of D2Q9 already grade
        assert got != ungraded

"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself:
printed values (Table 1, Fig. 2, Eq. PredictionWithMatrix under
tests/golden/), the recovery procedure of Appendix 2 in exact rationals,
polynomial exactness, consistency (Eq. ConsistencyPrediction), detail
redundancy (Eq. DetailRedundancy), the reduction of the adaptive step to the
reference scheme (Eq. StreamFinest) when epsilon = 0, a closed form of the
transport on a uniform coarse level, conservation, and a brute-force minimal
grading on tiny trees.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import Oracle, prediction_coefficient, predict_children
from paper_2103_02903_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------
# prediction operator
# ---------------------------------------------------------------------------

def _appendix2_weights(s):
    """Appendix 2: fit a degree-2s polynomial to 2s+1 cell means (unit cells
    centred at -s..s), then average it over the left child [-1/2, 0].
    Returns the weights of f_{-s..s} in the left-child prediction."""
    n = 2 * s + 1

    def mean_monomial(a, b, m):
        return (Fraction(b) ** (m + 1) - Fraction(a) ** (m + 1)) / ((m + 1) * (Fraction(b) - Fraction(a)))

    T = [[mean_monomial(Fraction(2 * k - 1, 2), Fraction(2 * k + 1, 2), m) for m in range(n)]
         for k in range(-s, s + 1)]
    # invert T exactly (Gauss-Jordan)
    A = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(T)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        inv = 1 / A[c][c]
        A[c] = [v * inv for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                fac = A[r][c]
                A[r] = [vr - fac * vc for vr, vc in zip(A[r], A[c])]
    Tinv = [row[n:] for row in A]
    child = [mean_monomial(Fraction(-1, 2), Fraction(0), m) for m in range(n)]
    return [sum(child[m] * Tinv[m][k] for m in range(n)) for k in range(n)]


@pytest.mark.parametrize("s", [1, 2, 3])
def test_table1_from_appendix2(s):
    rows = {int(r[0]): r[1:] for r in _read_rows("prediction_coefficients.txt")}
    printed = [Fraction(v) for v in rows[s] if v != "-"]
    w = _appendix2_weights(s)
    # left child: f_0 + sum_a c_a (f_a - f_-a)  => weight of f_a is c_a
    for a in range(1, s + 1):
        assert w[s + a] == printed[a - 1]
        assert w[s - a] == -printed[a - 1]
    assert w[s] == 1


def test_oracle_coefficient_is_table1():
    assert prediction_coefficient() == -0.125


def _impulse_weights(d, cross_sign, child=0):
    n = 3 ** d
    out = np.zeros(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        out[i] = predict_children(d, e, cross_sign)[child]
    return out


def test_fig2_weights_and_kronecker_reading():
    """Axis and parent weights match Fig. 2; the diagonal weights of the
    default operator are the Kronecker product of the 1D ones (Appendix 2),
    which is the negative of the printed diagonal signs; cross_sign=-1
    reproduces the printing exactly."""
    printed = {(int(r[0]), int(r[1])): float(Fraction(r[2]))
               for r in _read_rows("prediction_weights_2d_fig2.txt")}
    w_tensor = _impulse_weights(2, +1)
    w_printed = _impulse_weights(2, -1)
    w1 = [float(v) for v in _appendix2_weights(1)]  # weights of offsets -1, 0, +1
    for (ox, oy), val in printed.items():
        i = (oy + 1) * 3 + (ox + 1)
        assert w_printed[i] == val
        kron = w1[ox + 1] * w1[oy + 1]
        assert w_tensor[i] == kron
        if ox != 0 and oy != 0:
            assert w_tensor[i] == -val
        else:
            assert w_tensor[i] == val


def _cell_mean_poly(coef, lo, hi):
    """Mean of sum_k coef[k] x^k over [lo, hi]."""
    return sum(c * (hi ** (k + 1) - lo ** (k + 1)) / ((k + 1) * (hi - lo)) for k, c in enumerate(coef))


def _stencil_and_children(d, coefs):
    """Means of a separable sum of products of 1D polynomials on the 3^d
    parent stencil (unit cells centred at -1, 0, 1) and on the 2^d children."""
    def mean_box(lo, hi):
        tot = 0.0
        for term in coefs:  # term: list of d coefficient lists
            prod = 1.0
            for a in range(d):
                prod *= _cell_mean_poly(term[a], lo[a], hi[a])
            tot += prod
        return tot

    st = np.zeros(3 ** d)
    for idx in itertools.product(range(3), repeat=d):
        lo = [i - 1 - 0.5 for i in idx]
        hi = [i - 1 + 0.5 for i in idx]
        flat = sum(idx[a] * 3 ** a for a in range(d))
        st[flat] = mean_box(lo, hi)
    ch = np.zeros(2 ** d)
    for ci in range(2 ** d):
        dl = [(ci >> a) & 1 for a in range(d)]
        lo = [-0.5 + 0.5 * dl[a] for a in range(d)]
        hi = [0.0 + 0.5 * dl[a] for a in range(d)]
        ch[ci] = mean_box(lo, hi)
    return st, ch


@pytest.mark.parametrize("d", [1, 2, 3])
def test_prediction_exact_on_tensor_quadratics(d):
    rng = np.random.default_rng(d)
    for _ in range(5):
        coefs = [[list(rng.standard_normal(3)) for _ in range(d)] for _ in range(3)]
        st, ch = _stencil_and_children(d, coefs)
        pred = predict_children(d, st, +1)
        np.testing.assert_allclose(pred, ch, rtol=0, atol=1e-13)


def test_printed_cross_sign_not_exact_on_xy():
    """With the diagonal sign as printed, f(x, y) = x y is not reproduced
    (the paper's stated exactness for degree 2s fails); the default is exact."""
    st, ch = _stencil_and_children(2, [[[0.0, 1.0], [0.0, 1.0]]])
    np.testing.assert_allclose(predict_children(2, st, +1), ch, atol=1e-15)
    err = predict_children(2, st, -1) - ch
    assert np.abs(err).max() > 0.1


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("cross", [1, -1])
def test_consistency_projection_of_prediction(d, cross):
    rng = np.random.default_rng(10 + d)
    for _ in range(20):
        st = rng.standard_normal(3 ** d)
        centre = st[(3 ** d) // 2]
        pred = predict_children(d, st, cross)
        assert abs(pred.mean() - centre) <= 4 * np.finfo(float).eps * max(1.0, np.abs(st).max())
        dy = rng.integers(-64, 64, 3 ** d) / 1024.0  # dyadic: exact
        assert predict_children(d, dy, cross).mean() == dy[(3 ** d) // 2]


@pytest.mark.parametrize("d", [1, 2, 3])
def test_detail_redundancy(d):
    rng = np.random.default_rng(20 + d)
    for _ in range(20):
        st = rng.standard_normal(3 ** d)
        children = rng.standard_normal(2 ** d)
        st[(3 ** d) // 2] = children.mean()
        details = children - predict_children(d, st, +1)
        assert abs(details.sum()) < 1e-14


# ---------------------------------------------------------------------------
# reference scheme (epsilon = 0)
# ---------------------------------------------------------------------------

def _ref_scheme(cfg):
    """Velocities, moment matrix, relaxation and equilibria typed from the
    paper (Sec. 7) for the uniform reference solver of the tests."""
    lam = cfg["lambda_"]
    sch = cfg["scheme"]
    if sch in ("d1q2_advection", "d1q2_burgers"):
        eta = [(1,), (-1,)]
        M = np.array([[1, 1], [lam, -lam]], float)
        S = [[0, cfg["s"][0]]]
        V = cfg["phys"][0]
        meq = (lambda u: [[u[0], V * u[0]]]) if sch == "d1q2_advection" else (lambda u: [[u[0], 0.5 * u[0] ** 2]])
        cons = [(0, 0)]
        m = 1
    elif sch == "d3q6_advection":
        # Sec. 7.3: velocities +-e_x, +-e_y, +-e_z, M and S as printed
        eta = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
        L2 = lam * lam
        M = np.array([[1, 1, 1, 1, 1, 1], [lam, -lam, 0, 0, 0, 0], [0, 0, lam, -lam, 0, 0],
                      [0, 0, 0, 0, lam, -lam], [L2, L2, -L2, -L2, 0, 0], [L2, L2, 0, 0, -L2, -L2]], float)
        s1, s2 = cfg["s"][0], cfg["s"][1]
        S = [[0, s1, s1, s1, s2, s2]]
        Vx, Vy, Vz = cfg["phys"][0:3]
        meq = lambda u: [[u[0], Vx * u[0], Vy * u[0], Vz * u[0], 0.0 * u[0], 0.0 * u[0]]]
        cons = [(0, 0)]
        m = 1
    elif sch == "d1q3_shallow_water":
        eta = [(0,), (1,), (-1,)]
        M = np.array([[1, 1, 1], [0, lam, -lam], [0, lam ** 2, lam ** 2]], float)
        S = [[0, 0, cfg["s"][0]]]
        g = cfg["phys"][0]
        meq = lambda u: [[u[0], u[1], u[1] ** 2 / u[0] + 0.5 * g * u[0] ** 2]]
        cons = [(0, 0), (0, 1)]
        m = 1
    elif sch == "d2q4x4_euler":
        eta = [(1, 0), (0, 1), (-1, 0), (0, -1)]
        M = np.array([[1, 1, 1, 1], [lam, 0, -lam, 0], [0, lam, 0, -lam],
                      [lam ** 2, -lam ** 2, lam ** 2, -lam ** 2]], float)
        S = [[0, cfg["s"][i], cfg["s"][i], cfg["s"][4 + i]] for i in range(4)]
        gam = cfg["phys"][0]

        def meq(u):
            rho, mx, my, E = u
            vx, vy = mx / rho, my / rho
            p = (gam - 1) * (E - 0.5 * (mx * vx + my * vy))
            fx = [mx, mx * vx + p, my * vx, vx * (E + p)]
            fy = [my, mx * vy, my * vy + p, vy * (E + p)]
            return [[u[i], fx[i], fy[i], 0 * rho] for i in range(4)]
        cons = [(i, 0) for i in range(4)]
        m = 4
    elif sch == "d2q9_ns":
        eta = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
        L = lam
        M = np.array([
            [1] * 9,
            [0, L, 0, -L, 0, L, -L, -L, L],
            [0, 0, L, 0, -L, L, L, -L, -L],
            [-4 * L ** 2] + [-L ** 2] * 4 + [2 * L ** 2] * 4,
            [0, -2 * L ** 3, 0, 2 * L ** 3, 0, L ** 3, -L ** 3, -L ** 3, L ** 3],
            [0, 0, -2 * L ** 3, 0, 2 * L ** 3, L ** 3, L ** 3, -L ** 3, -L ** 3],
            [4 * L ** 4] + [-2 * L ** 4] * 4 + [L ** 4] * 4,
            [0, L ** 2, -L ** 2, L ** 2, -L ** 2, 0, 0, 0, 0],
            [0, 0, 0, 0, 0, L ** 2, -L ** 2, L ** 2, -L ** 2]], float)
        s1, s2 = cfg["s"][0], cfg["s"][1]
        S = [[0, 0, 0, s1, s1, s1, s1, s2, s2]]
        cs2 = L * L / 3

        def meq(u):
            rho, qx, qy = u
            q2 = qx * qx + qy * qy
            return [[rho, qx, qy, 3 * (-2 * cs2 * rho + q2 / rho), -3 * cs2 * qx, -3 * cs2 * qy,
                     9 * (cs2 * cs2 * rho - cs2 * q2 / rho), (qx * qx - qy * qy) / rho, qx * qy / rho]]
        cons = [(0, 0), (0, 1), (0, 2)]
        m = 1
    q = len(eta)
    return eta, M, np.linalg.inv(M), np.array(S, float), meq, cons, m, q


class _Ref:
    """Uniform finest-level reference scheme: Eq. StreamFinest with
    Eq. refBoundaryConditions, then Eq. CollisionOnFinest."""

    def __init__(self, cfg, conserved):
        self.cfg = cfg
        self.eta, self.M, self.Minv, self.S, self.meq, self.cons, self.m, self.q = _ref_scheme(cfg)
        self.d = len(self.eta[0])
        self.shape = tuple(cfg["roots"][a] << cfg["max_level"] for a in range(self.d))[::-1]  # (ny, nx)
        N = conserved.shape[1]
        u = [conserved[k].reshape(self.shape) for k in range(len(self.cons))]
        meq = self.meq(u)
        self.f = np.zeros((self.m * self.q,) + self.shape)
        for i in range(self.m):
            mi = np.stack([np.broadcast_to(np.asarray(meq[i][r], float), self.shape) for r in range(self.q)])
            self.f[i * self.q:(i + 1) * self.q] = np.tensordot(self.Minv, mi, axes=1)
        assert N == int(np.prod(self.shape))

    def _bc(self, face, fstar, p):
        kind = self.cfg["bc"][face]
        i, h = divmod(p, self.q)
        hd = [self.eta.index(tuple(-e for e in self.eta[k])) for k in range(self.q)][h]
        pd = i * self.q + hd
        if kind == "copy":
            return fstar[p]
        if kind == "bounce_back":
            return fstar[pd]
        if kind == "anti_bounce_back":
            return -fstar[pd]
        if kind == "bounce_back_velocity":
            rho0, ux, uy = self.cfg["phys"][0:3]
            meq = self.meq([np.asarray(rho0), np.asarray(rho0 * ux), np.asarray(rho0 * uy)])
            feq = self.Minv @ np.array([float(v) for v in meq[0]])
            return fstar[pd] + (feq[h] - feq[hd])
        raise ValueError(kind)

    def step(self):
        fs = self.f
        new = np.empty_like(fs)
        grids = np.meshgrid(*[np.arange(n) for n in self.shape], indexing="ij")  # (y, x)
        coords = grids[::-1]  # x, y
        Ns = self.shape[::-1]
        for p in range(self.m * self.q):
            e = self.eta[p % self.q]
            src = [coords[a] - e[a] for a in range(self.d)]
            face = np.full(self.shape, -1)
            for a in range(self.d):
                per = self.cfg["bc"][2 * a] == "periodic"
                if per:
                    src[a] = src[a] % Ns[a]
                else:
                    out_lo = (src[a] < 0) & (face < 0)
                    out_hi = (src[a] >= Ns[a]) & (face < 0)
                    face[out_lo] = 2 * a
                    face[out_hi] = 2 * a + 1
            inside = face < 0
            cl = [np.clip(src[a], 0, Ns[a] - 1) for a in range(self.d)]
            val = fs[p][tuple(cl[::-1])]
            for fc in range(2 * self.d):
                sel = face == fc
                if sel.any():
                    val = np.where(sel, self._bc(fc, fs, p), val)
            new[p] = np.where(inside, val, val)
        # collide
        mo = [np.tensordot(self.M, new[i * self.q:(i + 1) * self.q], axes=1) for i in range(self.m)]
        u = [mo[li][mi] for (li, mi) in self.cons]
        meq = self.meq(u)
        for i in range(self.m):
            for r in range(self.q):
                s = self.S[i][r]
                mo[i][r] = (1 - s) * mo[i][r] + s * np.asarray(meq[i][r], float)
            new[i * self.q:(i + 1) * self.q] = np.tensordot(self.Minv, mo[i], axes=1)
        self.f = new


def _leaves_dense(o):
    lev, ix, iy, iz, f = o.leaves()
    assert (lev == o.J).all()
    shape = o.level_shape(o.J)
    if o.d == 3:
        idx = (iz.astype(np.int64) * shape[1] + iy) * shape[0] + ix
    elif o.d == 2:
        idx = iy.astype(np.int64) * shape[0] + ix
    else:
        idx = ix.astype(np.int64)
    out = np.zeros((o.Q, int(np.prod(shape))))
    out[:, idx] = f
    return out


@pytest.mark.parametrize("name,kw,steps", [
    ("advection_1d", dict(max_level=7), 20),
    ("burgers_1d", dict(max_level=7), 20),
    ("shallow_water_1d", dict(max_level=7), 20),
    ("euler_2d", dict(max_level=5), 8),
    ("ns_obstacle_2d", dict(max_level=4), 8),
    ("advection_3d", dict(max_level=4), 6),
])
def test_epsilon_zero_is_reference_scheme(name, kw, steps):
    cfg, u = W.WORKLOADS[name](seed=3, **kw)
    cfg["eps"] = 0.0
    cfg["obstacle"] = 0
    o = Oracle(cfg)
    o.init(u)
    ref = _Ref(cfg, u)
    for _ in range(steps):
        o.step(1)
        ref.step()
    got = _leaves_dense(o)
    want = ref.f.reshape(ref.f.shape[0], -1)
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


def test_equilibrium_of_constant_state_is_fixed():
    cfg, u = W.euler_2d(seed=1, max_level=5)
    u[:] = u[:, :1]  # constant state
    o = Oracle(cfg)
    o.init(u)
    f0 = o.leaves()[4][:, 0].copy()
    o.step(3)
    f = o.leaves()[4]
    np.testing.assert_allclose(f, f0[:, None] * np.ones_like(f), rtol=1e-13, atol=1e-13)


def test_relaxation_one_reaches_equilibrium_moment():
    cfg, u = W.advection_1d(seed=2, max_level=7)
    o = Oracle(cfg)
    o.init(u)
    o.step(5)
    f = o.leaves()[4]
    lam, V = cfg["lambda_"], cfg["phys"][0]
    np.testing.assert_allclose(lam * (f[0] - f[1]), V * (f[0] + f[1]), rtol=0, atol=1e-14)


@pytest.mark.parametrize("name,kw", [("advection_1d", dict(max_level=9)),
                                     ("euler_2d", dict(max_level=6)),
                                     ("ns_obstacle_2d", dict(max_level=5)),
                                     ("advection_3d", dict(max_level=5))])
def test_conservation_periodic(name, kw):
    cfg, u = W.WORKLOADS[name](seed=4, **kw)
    cfg["bc"] = ["periodic"] * 6
    cfg["obstacle"] = 0
    o = Oracle(cfg)
    o.init(u)
    J = cfg["max_level"]
    tot0 = o.project(J).sum(axis=1)
    o.step(12)
    tot = o.project(J).sum(axis=1)
    np.testing.assert_allclose(tot, tot0, rtol=1e-13, atol=1e-13 * np.abs(tot0).max())
    assert o.graded()


# ---------------------------------------------------------------------------
# transport on a uniform coarse level
# ---------------------------------------------------------------------------

def _uniform_state(cfg, level, rng):
    o = Oracle(cfg)
    n = cfg["roots"][0] << level
    lev = np.full(n, level, np.int32)
    ix = np.arange(n, dtype=np.int32)
    z = np.zeros(n, np.int32)
    f = rng.standard_normal((o.Q, n))
    o.set_leaves(lev, ix, z, z, f)
    return o, f


def test_uniform_coarse_level_closed_form():
    """All leaves at level J-1 (periodic D1Q2): the transport of Eq.
    AdaptiveAdvectionPhase reduces to
    f_k + 1/2 [f_{k-1} - f_k + (f_k + f_{k-1} - f_{k-2} - f_{k+1})/8] for eta = +1
    (and the mirror formula for eta = -1), derived from the s = 1 prediction."""
    cfg, _ = W.advection_1d(seed=0, max_level=7)
    rng = np.random.default_rng(5)
    o, f = _uniform_state(cfg, cfg["max_level"] - 1, rng)
    o.stream_collide(collide=False)
    got = o.leaves()[4]
    r = lambda a, k: np.roll(a, -k)  # r(a, k)[i] = a[i + k]
    fp = f[0]
    want_p = fp + 0.5 * (r(fp, -1) - fp + (fp + r(fp, -1) - r(fp, -2) - r(fp, 1)) / 8)
    fm = f[1]
    want_m = fm + 0.5 * (r(fm, 1) - fm + (fm + r(fm, 1) - r(fm, 2) - r(fm, -1)) / 8)
    np.testing.assert_allclose(got[0], want_p, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(got[1], want_m, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("gap", [1, 2, 3, 4])
def test_flattening_matrix_eq_prediction_with_matrix(gap):
    Mrows = [[Fraction(v) for v in row] for row in _read_rows("flattening_matrix_1d.txt")]
    Mf = np.array([[float(v) for v in row] for row in Mrows])
    cfg, _ = W.advection_1d(seed=0, max_level=8)
    rng = np.random.default_rng(gap)
    j = cfg["max_level"] - gap
    o, f = _uniform_state(cfg, j, rng)
    fine = o.reconstruct(cfg["max_level"])[0]
    P = np.linalg.matrix_power(Mf, gap)
    n = f.shape[1]
    w = 1 << gap
    for k in range(2, n - 2):
        want = P @ f[0, k - 2:k + 2]
        got = fine[w * k - 2:w * k + 2]
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------
# mesh adaptation: brute-force minimal grading on tiny 1D trees
# ---------------------------------------------------------------------------

def _all_trees_1d(Jmin, J, nroots):
    """Every tree (as the set of refined cells) over nroots level-Jmin roots."""
    def subtrees(level, k):
        if level == J:
            return [frozenset()]
        out = [frozenset()]
        left = subtrees(level + 1, 2 * k)
        right = subtrees(level + 1, 2 * k + 1)
        for a in left:
            for b in right:
                out.append(frozenset({(level, k)}) | a | b)
        return out
    per_root = [subtrees(Jmin, k) for k in range(nroots)]
    for combo in itertools.product(*per_root):
        yield frozenset().union(*combo)


def _cells_of(refined, Jmin, nroots):
    cells = {(Jmin, k) for k in range(nroots)}
    for (l, k) in refined:
        cells |= {(l + 1, 2 * k), (l + 1, 2 * k + 1)}
    return cells


def _graded(refined, Jmin, nroots, periodic=True):
    cells = _cells_of(refined, Jmin, nroots)
    for (l, k) in cells:
        if l == Jmin:
            continue
        n = 1 << (l - 1)  # roots = 1: 2^l cells at level l
        for o in (-1, 0, 1):
            c = k // 2 + o
            if periodic:
                c %= n
            elif c < 0 or c >= n:
                continue
            if (l - 1, c) not in cells:
                return False
    return True


@pytest.mark.parametrize("seed", range(6))
def test_adaptation_matches_brute_force_grading(seed):
    Jmin, J = 2, 4
    nroots = 1 << Jmin
    cfg, _ = W.advection_1d(seed=seed, max_level=J, min_level=Jmin, eps=3e-2)
    rng = np.random.default_rng(100 + seed)
    trees = list(_all_trees_1d(Jmin, J, 1))
    # start from a random graded tree with random data
    while True:
        refined = frozenset().union(*[frozenset((l, k + r * (1 << (l - Jmin))) for (l, k) in
                                                trees[rng.integers(len(trees))]) for r in range(nroots)])
        if _graded(refined, Jmin, nroots):
            break
    cells = _cells_of(refined, Jmin, nroots)
    leaves = sorted(c for c in cells if c not in refined)
    o = Oracle(cfg)
    lev = np.array([c[0] for c in leaves], np.int32)
    ix = np.array([c[1] for c in leaves], np.int32)
    z = np.zeros(len(leaves), np.int32)
    xs = (ix + 0.5) / (1 << lev)
    f = np.stack([np.where(xs < 0.4, 1.0, 0.2) + 0.3 * np.sin(7 * xs) + 0.02 * rng.standard_normal(len(xs)),
                  0.5 + 0.1 * np.cos(5 * xs)])
    o.set_leaves(lev, ix, z, z, f)
    assert o.graded()
    G = {}
    o.adapt()
    for l in range(Jmin, J):
        G[l] = o.group_norms(l)
    new_lev, new_ix = o.leaves()[0], o.leaves()[1]
    got = set(zip(new_lev.tolist(), new_ix.tolist()))

    # T_eps with closure, then H_eps, written from the set definitions
    d, eps, mu = 1, cfg["eps"], cfg["mu_bar"]
    epsl = lambda l: eps * 2.0 ** (d * (l - J))
    old_cells = cells

    def close(cellset):
        out = set(cellset) | {(Jmin, k) for k in range(nroots)}
        for (l, k) in list(out):
            while l > Jmin:
                p = k // 2
                out |= {(l, 2 * p), (l, 2 * p + 1)}
                l, k = l - 1, p
                out.add((l, k))
        return out

    T = close({(l, k) for (l, k) in old_cells if l > Jmin and G[l - 1][k // 2] >= epsl(l)})
    H = set(T)
    for (l, k) in T:
        n = 1 << l
        for e in (1, -1):
            H |= close({(l, (k - e) % n)})
        if Jmin < l < J and G[l - 1][k // 2] >= 2.0 ** (mu + d) * epsl(l):
            H |= close({(l + 1, 2 * k), (l + 1, 2 * k + 1)})
    # brute force: smallest graded tree containing H
    best = None
    allt = _all_trees_1d(Jmin, J, nroots)
    for ref in allt:
        cs = _cells_of(ref, Jmin, nroots)
        if not H <= cs or not _graded(ref, Jmin, nroots):
            continue
        if best is None or len(cs) < len(best):
            best = cs
    want = {c for c in best if (c[0] == J or (c[0] + 1, 2 * c[1]) not in best)}
    assert got == want
    assert o.graded()


def test_error_control_shape():
    """Additional error of Eq. AdditionalErrorEstimate decreases with epsilon
    (shape only: the paper gives no numbers)."""
    errs = []
    for eps in (1e-2, 1e-3, 1e-4):
        cfg, u = W.advection_1d(seed=0, max_level=9, eps=eps)
        o = Oracle(cfg)
        o.init(u)
        cfg0 = dict(cfg, eps=0.0)
        r = Oracle(cfg0)
        r.init(u)
        o.step(35)
        r.step(35)
        J = cfg["max_level"]
        a, b = o.project(J)[0], r.project(J)[0]
        errs.append(np.abs(a - b).sum() / np.abs(b).sum())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 5e-3

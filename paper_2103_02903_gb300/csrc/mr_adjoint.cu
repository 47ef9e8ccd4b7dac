// Adjoint of the time step of Algorithm 1 with the mesh of every step frozen
// (replayed from the forward pass).  For a given pair of meshes (M_n, M_n+1)
// the data transfer (Sec. 5.1), the ghost prediction (Sec. 4.1), the
// projection (Def. Projection) and the leaf-reconstruction transport
// (Eq. AdaptiveAdvectionPhase, Eq. AdvectionOnBoundary) are linear in the
// leaf values, so their adjoints are the transposed scatters below: every
// term "coefficient x value of a cell" of the forward operator sends
// "coefficient x adjoint of the output" to the adjoint of that cell.  The
// collision (Eq. AdaptiveCollision) and the obstacle penalisation are local:
// their Jacobians, with respect to the populations and to the relaxation
// rates, come from the same scheme code evaluated on dual numbers.
//
// All adjoint arithmetic is FP64.  Adjoint arrays have the layout of the
// value arrays ([Q][capacity] per cell class).
#include "mr_schemes.cuh"

namespace {

// ------------------------------------------------------------------ dual numbers
// Forward-mode derivatives with respect to N of the independent variables,
// the variables OFF .. OFF + N - 1 of a numbering in which 0 .. Q - 1 are
// the populations and Q + i is the relaxation rate s[i].
template <int N, int Q = 0, int OFF = 0>
struct Dual {
  double v;
  double d[N];
  __device__ Dual() {}
  __device__ Dual(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.0;
  }
};
#define MR_DUAL template <int N, int Q, int OFF>
#define MR_DT Dual<N, Q, OFF>
MR_DUAL __device__ __forceinline__ MR_DT operator+(const MR_DT& a, const MR_DT& b) {
  MR_DT r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
MR_DUAL __device__ __forceinline__ MR_DT operator-(const MR_DT& a, const MR_DT& b) {
  MR_DT r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
MR_DUAL __device__ __forceinline__ MR_DT operator-(const MR_DT& a) {
  MR_DT r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
MR_DUAL __device__ __forceinline__ MR_DT operator*(const MR_DT& a, const MR_DT& b) {
  MR_DT r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
MR_DUAL __device__ __forceinline__ MR_DT operator/(const MR_DT& a, const MR_DT& b) {
  MR_DT r;
  const double ib = 1.0 / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}

// a relaxation rate, seeded when it is one of the dual's variables
MR_DUAL struct RateOf<MR_DT> {
  __device__ static MR_DT get(const Geo& g, int i) {
    MR_DT r(g.s[i]);
    const int k = Q + i - OFF;
    if (k >= 0 && k < N) r.d[k] = 1.0;
    return r;
  }
};

// ------------------------------------------------------------------ cells
__device__ __forceinline__ double* adj_of(const Geo& g, double* aL, double* aI, double* aG, int32_t e) {
  const uint32_t cls = ((uint32_t)e) >> 30, idx = (uint32_t)e & 0x3FFFFFFFu;
  if (cls == MR_CLS_LEAF) return aL + idx;
  if (cls == MR_CLS_INT) return aI + idx;
  return aG + idx;
}
__device__ __forceinline__ size_t stride_of(const Geo& g, int32_t e) {
  const uint32_t cls = ((uint32_t)e) >> 30;
  return cls == MR_CLS_LEAF ? g.cap[0] : (cls == MR_CLS_INT ? g.cap[1] : g.cap[2]);
}

// ------------------------------------------------------------------ transport terms
// Enumerates the linear terms of the transport of leaf i of mesh B, in the
// order of the forward kernel: out[p] = sum of coef x value(cell, p_in).
// op.self(p, p_in, coef): a value of the leaf itself; op.cell(p, entry,
// p_in, coef): a value of another cell (index-map entry).  The constant of
// the moving-wall bounce back is not a term.
template <class Sc, class Op>
__device__ void bc_terms(const Geo& g, int kind, int p, double coef, Op& op) {
  switch (kind) {
    case 1: op.self(p, p, coef); break;
    case 2:
    case 4: op.self(p, Sc::opp(p), coef); break;
    case 3: op.self(p, Sc::opp(p), -coef); break;
    default: break;
  }
}

template <class Sc, class Op>
__device__ void transport_terms(const Geo& g, const MeshDev& B, const double* __restrict__ W, int i, Op& op) {
  constexpr int D = Sc::D, Q = Sc::Q;
  const int l = B.lvl[MR_CLS_LEAF][i];
  int x, y;
  mr_decode(g, l, B.code[MR_CLS_LEAF][i], x, y);
  const double scale = ldexp(1.0, l - g.J);
  const double cs = (double)g.cross_sign;
  for (int p = 0; p < Q; ++p) op.self(p, p, 1.0);
  for (int a = 0; a < D; ++a) {
    const int k = a == 0 ? x : y;
    const int N = g.n[l][a], per = g.periodic[a];
    const int slot = mr_slot(k, N, per);
    const double* wP = W + MR_WIDX(l, a, slot, 0);
    const double* wM = W + MR_WIDX(l, a, slot, 1);
    int32_t ent[4];
    bool has[4];
    for (int w = 0; w < 4; ++w) {
      const int off = w < 2 ? w - 2 : w - 1;
      int nx = x + (a == 0 ? off : 0), ny = y + (a == 1 ? off : 0);
      has[w] = mr_nbr_mesh(g, l, nx, ny);
      ent[w] = has[w] ? B.map[g.base[l] + mr_encode(g, l, nx, ny)] : MR_MAP_NONE;
      if (has[w] && ent[w] == MR_MAP_NONE) {
        mr_set_err(B.cnt, MR_DERR_INTERNAL);
        has[w] = false;
      }
    }
    for (int p = 0; p < Q; ++p) {
      const int sgn = eta_of<Sc>(p, a);
      if (sgn == 0) continue;
      const double* w = sgn > 0 ? wP : wM;
      op.self(p, p, scale * w[2]);
      for (int q = 0; q < 4; ++q)
        if (has[q]) op.cell(p, ent[q], p, scale * w[q < 2 ? q : q + 1]);
      if (!per) {
        if (sgn > 0 && k == 0) bc_terms<Sc>(g, g.bc[2 * a], p, scale, op);
        if (sgn < 0 && k == N - 1) bc_terms<Sc>(g, g.bc[2 * a + 1], p, scale, op);
      }
    }
    // refined neighbour on either side along a: one-level detail correction
    for (int side = -1; side <= 1; side += 2) {
      const int wi = side < 0 ? 1 : 2;
      if (!has[wi] || (((uint32_t)ent[wi]) >> 30) != MR_CLS_INT) continue;
      int nx = x + (a == 0 ? side : 0), ny = y + (a == 1 ? side : 0);
      mr_nbr_mesh(g, l, nx, ny);
      int32_t st[9], ce[1 << D];
      bool ok = mr_stencil_entries<D>(g, B, l, nx, ny, st);
      const uint32_t ncode = mr_encode(g, l, nx, ny);
      for (int ci = 0; ci < (1 << D); ++ci) {
        ce[ci] = B.map[g.base[l + 1] + ((ncode << D) | (uint32_t)ci)];
        ok = ok && ce[ci] != MR_MAP_NONE;
      }
      if (!ok) {
        mr_set_err(B.cnt, MR_DERR_INTERNAL);
        continue;
      }
      const int N1 = g.n[l + 1][a];
      for (int p = 0; p < Q; ++p) {
        const int sgn = eta_of<Sc>(p, a);
        if (sgn == 0) continue;
        const bool incoming = (sgn > 0) == (side < 0);
        int c;
        if (sgn > 0)
          c = side < 0 ? 2 * k - 1 : 2 * k + 1;
        else
          c = side > 0 ? 2 * k + 2 : 2 * k;
        const int cslot = mr_slot(per ? 2 : c, N1, per);
        const double* wt = W + MR_WIDX(l + 1, a, cslot, sgn > 0 ? 2 : 3);
        const double factor = (D == 2 ? 0.5 : 1.0) * scale * (incoming ? 1.0 : -1.0);
        for (int ci = 0; ci < (1 << D); ++ci) {
          const int sa = (ci >> a) & 1;
          const int delta = 2 * (k + side) + sa - c;
          if (delta < -2 || delta > 2) continue;
          const double cw = wt[delta + 2] * factor;
          op.cell(p, ce[ci], p, cw);
          double pw[9];
          predict_weights<D>(ci, cs, pw);
          for (int kk = 0; kk < (D == 2 ? 9 : 3); ++kk) op.cell(p, st[kk], p, -cw * pw[kk]);
        }
      }
    }
  }
  if constexpr (Sc::DIAG) {
    // corner cells of the diagonal velocities (see the forward transport)
    constexpr int P0 = Sc::DIAG0;
    const double scale2 = scale * scale;
    const int Nx = g.n[l][0], Ny = g.n[l][1];
    const int slx = mr_slot(x, Nx, g.periodic[0]), sly = mr_slot(y, Ny, g.periodic[1]);
    const double* wx[2] = {W + MR_WIDX(l, 0, slx, 0), W + MR_WIDX(l, 0, slx, 1)};
    const double* wy[2] = {W + MR_WIDX(l, 1, sly, 0), W + MR_WIDX(l, 1, sly, 1)};
    for (int b = 0; b < 5; ++b)
      for (int a = 0; a < 5; ++a) {
        const bool self = a == 2 && b == 2;
        int32_t e = MR_MAP_NONE;
        if (!self) {
          int nx = x + a - 2, ny = y + b - 2;
          if (!mr_nbr_mesh(g, l, nx, ny)) continue;
          e = B.map[g.base[l] + mr_encode(g, l, nx, ny)];
          if (e == MR_MAP_NONE) {
            mr_set_err(B.cnt, MR_DERR_INTERNAL);
            continue;
          }
        }
        for (int t = 0; t < 4; ++t) {
          const int p = P0 + t;
          const double wab = wx[Sc::eta(p, 0) > 0 ? 0 : 1][a] * wy[Sc::eta(p, 1) > 0 ? 0 : 1][b];
          if (self)
            op.self(p, p, scale2 * wab);
          else
            op.cell(p, e, p, scale2 * wab);
        }
      }
    if (l < g.J) {
      for (int nb = 0; nb < 9; ++nb) {
        if (nb == 4) continue;
        const int dx = nb % 3 - 1, dy = nb / 3 - 1;
        int nx = x + dx, ny = y + dy;
        if (!mr_nbr_mesh(g, l, nx, ny)) continue;
        const uint32_t ncode = mr_encode(g, l, nx, ny);
        const int32_t e = B.map[g.base[l] + ncode];
        if (e == MR_MAP_NONE || (((uint32_t)e) >> 30) != MR_CLS_INT) continue;
        int32_t st[9], ce[4];
        bool ok = mr_stencil_entries<2>(g, B, l, nx, ny, st);
        for (int ci = 0; ci < 4; ++ci) {
          ce[ci] = B.map[g.base[l + 1] + ((ncode << 2) | (uint32_t)ci)];
          ok = ok && ce[ci] != MR_MAP_NONE;
        }
        if (!ok) {
          mr_set_err(B.cnt, MR_DERR_INTERNAL);
          continue;
        }
        for (int t = 0; t < 4; ++t) {
          const int p = P0 + t;
          const int sx = Sc::eta(p, 0), sy = Sc::eta(p, 1);
          for (int ci = 0; ci < 4; ++ci) {
            const double w = corner_edge_weight<double>(g, W, l + 1, 0, x, 2 * dx + (ci & 1), sx) *
                             corner_edge_weight<double>(g, W, l + 1, 1, y, 2 * dy + (ci >> 1), sy);
            if (w == 0.0) continue;
            op.cell(p, ce[ci], p, scale2 * w);
            double pw[9];
            predict_weights<2>(ci, cs, pw);
            for (int kk = 0; kk < 9; ++kk) op.cell(p, st[kk], p, -scale2 * w * pw[kk]);
          }
        }
      }
    }
    for (int t = 0; t < 4; ++t) {
      const int p = P0 + t;
      const int sx = Sc::eta(p, 0), sy = Sc::eta(p, 1);
      const bool outx = !g.periodic[0] && (sx > 0 ? x == 0 : x == Nx - 1);
      const bool outy = !g.periodic[1] && (sy > 0 ? y == 0 : y == Ny - 1);
      if (outx && outy) bc_terms<Sc>(g, g.bc[sy > 0 ? 2 : 3], p, -scale2, op);
    }
  }
}

// ------------------------------------------------------------------ collision
// Jacobian-transpose products of collision + obstacle for the variables
// OFF .. OFF + 7 (populations, then rates), then the next chunk.
template <int SC, int OFF>
__device__ void adj_collide_chunk(const Geo& g, double phi, const double* z, const double* lm, double* mu,
                                  double* dsl) {
  using Sc = Scheme<SC>;
  constexpr int Q = Sc::Q, NV = Q + Sc::NR;
  using T = Dual<8, Q, OFF>;
  T f[Q];
#pragma unroll
  for (int p = 0; p < Q; ++p) {
    f[p] = T(z[p]);
    if (p >= OFF && p < OFF + 8) f[p].d[p - OFF] = 1.0;
  }
  Sc::template collide<T>(g, f);
  if (phi > 0.0)
    for (int p = 0; p < Q; ++p) f[p] = T(phi * g.feq0[p]) + T(1.0 - phi) * f[p];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int var = OFF + k;
    if (var >= NV) break;
    double s = 0;
#pragma unroll
    for (int p = 0; p < Q; ++p) s += lm[p] * f[p].d[k];
    if (var < Q)
      mu[var] = s;
    else
      dsl[var - Q] += s;
  }
  if constexpr (OFF + 8 < NV) adj_collide_chunk<SC, OFF + 8>(g, phi, z, lm, mu, dsl);
}

// Leaves of M_n+1.  In: lam = d J / d x_n+1 (adjoint of the stored state).
// Adds the functional's own term at x_n+1 when `source`, takes the adjoint
// through the obstacle and the collision at the pre-collision state z, and
// leaves d J / d z in lam; the rates' part is summed into ds[16].
template <int SC>
__global__ void __launch_bounds__(128) k_adj_collide(Geo g, MeshDev B, const double* __restrict__ z, double* lam,
                                                     double* ds, int source, double vol_J) {
  using Sc = Scheme<SC>;
  constexpr int Q = Sc::Q;
  const int n = B.cnt->total[MR_CLS_LEAF];
  double dsl[16];
  for (int r = 0; r < 16; ++r) dsl[r] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int l = B.lvl[MR_CLS_LEAF][i];
    const uint32_t code = B.code[MR_CLS_LEAF][i];
    double zi[Q], x[Q], lm[Q], mu[Q];
    for (int p = 0; p < Q; ++p) x[p] = zi[p] = z[(size_t)p * g.cap[0] + i];
    Sc::template collide<double>(g, x);
    double phi = 0.0;
    if constexpr (Sc::DIAG) {
      if (g.obstacle) phi = obstacle_fraction(g, l, code);
      if (phi > 0.0)
        for (int p = 0; p < Q; ++p) x[p] = phi * g.feq0[p] + (1.0 - phi) * x[p];
    }
    for (int p = 0; p < Q; ++p) lm[p] = lam[(size_t)p * g.cap[0] + i];
    if (source) {
      // kinetic energy vol |q|^2 / (2 rho) of the state after the step
      double u[4] = {0, 0, 0, 0};
      for (int k = 0; k < g.ncons; ++k)
        for (int p = 0; p < Q; ++p) u[k] += g.consw[k][p] * x[p];
      const double vol = vol_J * ldexp(1.0, g.d * (g.J - l));
      double du[4] = {0, 0, 0, 0};
      if (g.ncons == 1) {
        du[0] = u[0];
      } else {
        double q2 = 0;
        for (int k = 1; k < g.ncons && k < 3; ++k) q2 += u[k] * u[k];
        du[0] = -0.5 * q2 / (u[0] * u[0]);
        for (int k = 1; k < g.ncons && k < 3; ++k) du[k] = u[k] / u[0];
      }
      for (int p = 0; p < Q; ++p) {
        double s = 0;
        for (int k = 0; k < g.ncons; ++k) s += du[k] * g.consw[k][p];
        lm[p] += vol * s;
      }
    }
    adj_collide_chunk<SC, 0>(g, phi, zi, lm, mu, dsl);
    for (int p = 0; p < Q; ++p) lam[(size_t)p * g.cap[0] + i] = mu[p];
  }
  // rates: warp sums, one atomic per warp and rate
  for (int r = 0; r < 16; ++r) {
    double v = dsl[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&ds[r], v);
  }
}

// Transport: scatter coef x adjoint(out) into the adjoints of the cells read.
template <int SC>
__global__ void __launch_bounds__(128) k_adj_transport(Geo g, MeshDev B, const double* __restrict__ W,
                                                       const double* __restrict__ mu, double* aL, double* aI,
                                                       double* aG) {
  using Sc = Scheme<SC>;
  constexpr int Q = Sc::Q;
  const int n = B.cnt->total[MR_CLS_LEAF];
  struct Scatter {
    const Geo& g;
    double *aL, *aI, *aG;
    int i;
    double m[Q];
    __device__ void self(int p, int pin, double c) { atomicAdd(aL + (size_t)pin * g.cap[0] + i, c * m[p]); }
    __device__ void cell(int p, int32_t e, int pin, double c) {
      atomicAdd(adj_of(g, aL, aI, aG, e) + (size_t)pin * stride_of(g, e), c * m[p]);
    }
  };
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    Scatter op{g, aL, aI, aG, i, {}};
    bool any = false;
    for (int p = 0; p < Q; ++p) {
      op.m[p] = mu[(size_t)p * g.cap[0] + i];
      any = any || op.m[p] != 0.0;
    }
    if (any) transport_terms<Sc>(g, B, W, i, op);
  }
}

// Ghost / created-leaf prediction of one level, transposed: the adjoint of a
// predicted cell goes to its stencil on level - 1 (levels fine to coarse).
template <int D, int Q>
__global__ void __launch_bounds__(128) k_adj_predict(Geo g, MeshDev B, int level, double* aL, double* aI,
                                                     double* aG) {
  const int gb = B.cnt->off[MR_CLS_GHOST][level], ng = B.cnt->off[MR_CLS_GHOST][level + 1] - gb;
  const int lb = B.cnt->off[MR_CLS_LEAF][level], nl = B.cnt->off[MR_CLS_LEAF][level + 1] - lb;
  const double cs = (double)g.cross_sign;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ng + nl; t += gridDim.x * blockDim.x) {
    uint32_t code;
    const double* a;
    size_t as;
    if (t < ng) {
      code = B.code[MR_CLS_GHOST][gb + t];
      a = aG + gb + t;
      as = g.cap[2];
    } else {
      const int i = lb + (t - ng);
      if (B.src[i] >= 0) continue;  // copied, not predicted
      code = B.code[MR_CLS_LEAF][i];
      a = aL + i;
      as = g.cap[0];
    }
    int px, py;
    mr_decode(g, level - 1, code >> D, px, py);
    int32_t st[9];
    if (!mr_stencil_entries<D>(g, B, level - 1, px, py, st)) {
      mr_set_err(B.cnt, MR_DERR_INTERNAL);
      continue;
    }
    double pw[9];
    predict_weights<D>((int)(code & ((1u << D) - 1u)), cs, pw);
    for (int p = 0; p < Q; ++p) {
      const double v = a[(size_t)p * as];
      if (v == 0.0) continue;
      for (int kk = 0; kk < (D == 2 ? 9 : 3); ++kk)
        atomicAdd(adj_of(g, aL, aI, aG, st[kk]) + (size_t)p * stride_of(g, st[kk]), pw[kk] * v);
    }
  }
}

// Data transfer transposed: a copied leaf or internal cell of M_n+1 hands its
// adjoint to the cell of M_n it was copied from.
template <int Q>
__global__ void __launch_bounds__(128) k_adj_transfer(Geo g, MeshDev A, MeshDev B, const double* __restrict__ aLB,
                                                      const double* __restrict__ aIB, double* aLA, double* aIA) {
  const int nL = B.cnt->total[MR_CLS_LEAF], nI = B.cnt->total[MR_CLS_INT];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nL + nI; t += gridDim.x * blockDim.x) {
    const bool leaf = t < nL;
    const int i = leaf ? t : t - nL;
    const int k = leaf ? MR_CLS_LEAF : MR_CLS_INT;
    if (leaf && B.src[i] < 0) continue;
    const int32_t e = A.map[g.base[B.lvl[k][i]] + B.code[k][i]];
    if (e == MR_MAP_NONE || (((uint32_t)e) >> 30) > MR_CLS_INT) continue;
    const double* src = leaf ? aLB + i : aIB + i;
    const size_t ss = leaf ? g.cap[0] : g.cap[1];
    double* dst = (((uint32_t)e) >> 30) == MR_CLS_LEAF ? aLA + ((uint32_t)e & 0x3FFFFFFFu)
                                                       : aIA + ((uint32_t)e & 0x3FFFFFFFu);
    const size_t ds = (((uint32_t)e) >> 30) == MR_CLS_LEAF ? g.cap[0] : g.cap[1];
    for (int p = 0; p < Q; ++p) atomicAdd(dst + (size_t)p * ds, src[(size_t)p * ss]);
  }
}

// Projection transposed (levels coarse to fine): an internal cell of M_n
// hands 2^-d of its adjoint to each child.
template <int D, int Q>
__global__ void __launch_bounds__(128) k_adj_project(Geo g, MeshDev A, int level, double* aLA, double* aIA) {
  const int b0 = A.cnt->off[MR_CLS_INT][level], b1 = A.cnt->off[MR_CLS_INT][level + 1];
  const double scale = D == 1 ? 0.5 : 0.25;
  for (int i = b0 + blockIdx.x * blockDim.x + threadIdx.x; i < b1; i += gridDim.x * blockDim.x) {
    const uint32_t code = A.code[MR_CLS_INT][i];
    for (int ci = 0; ci < (1 << D); ++ci) {
      const int32_t e = A.map[g.base[level + 1] + ((code << D) | (uint32_t)ci)];
      if (e == MR_MAP_NONE || (((uint32_t)e) >> 30) > MR_CLS_INT) {
        mr_set_err(A.cnt, MR_DERR_INTERNAL);
        continue;
      }
      const bool lf = (((uint32_t)e) >> 30) == MR_CLS_LEAF;
      double* dst = (lf ? aLA : aIA) + ((uint32_t)e & 0x3FFFFFFFu);
      const size_t ds = lf ? g.cap[0] : g.cap[1];
      for (int p = 0; p < Q; ++p) atomicAdd(dst + (size_t)p * ds, scale * aIA[(size_t)p * g.cap[1] + i]);
    }
  }
}

// Initial state: f = M^-1 m^eq(u0) on the full finest mesh; d J / d u0 from
// the equilibrium's Jacobian (dual numbers in the conserved moments).
template <int SC>
__global__ void __launch_bounds__(128) k_adj_init(Geo g, MeshDev B, const double* __restrict__ cons,
                                                  const double* __restrict__ lam, double* grad) {
  using Sc = Scheme<SC>;
  constexpr int Q = Sc::Q;
  const int n = B.cnt->total[MR_CLS_LEAF];
  const long long NJ = (long long)g.n[g.J][0] * (Sc::D == 2 ? g.n[g.J][1] : 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int x, y;
    mr_decode(g, g.J, B.code[MR_CLS_LEAF][i], x, y);
    const long long r = (long long)y * g.n[g.J][0] + x;
    using T = Dual<4>;
    T u[4], f[Q];
    for (int k = 0; k < 4; ++k) {
      u[k] = T(k < g.ncons ? cons[k * NJ + r] : 0.0);
      u[k].d[k] = 1.0;
    }
    Sc::template equilibrium<T>(g, u, f);
    for (int k = 0; k < g.ncons; ++k) {
      double s = 0;
      for (int p = 0; p < Q; ++p) s += lam[(size_t)p * g.cap[0] + i] * f[p].d[k];
      grad[k * NJ + r] = s;
    }
  }
}

// Functional of a state: sum over leaves of vol |q|^2 / (2 rho) (1/2 u^2
// for a single conserved moment), added to *J.
template <int SC>
__global__ void __launch_bounds__(128) k_kinetic_energy(Geo g, MeshDev B, const double* __restrict__ LF,
                                                        double vol_J, double* J) {
  using Sc = Scheme<SC>;
  constexpr int Q = Sc::Q;
  const int n = B.cnt->total[MR_CLS_LEAF];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double u[4] = {0, 0, 0, 0};
    for (int k = 0; k < g.ncons; ++k)
      for (int p = 0; p < Q; ++p) u[k] += g.consw[k][p] * LF[(size_t)p * g.cap[0] + i];
    double e;
    if (g.ncons == 1) {
      e = 0.5 * u[0] * u[0];
    } else {
      double q2 = 0;
      for (int k = 1; k < g.ncons && k < 3; ++k) q2 += u[k] * u[k];
      e = 0.5 * q2 / u[0];
    }
    acc += vol_J * ldexp(1.0, g.d * (g.J - B.lvl[MR_CLS_LEAF][i])) * e;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(J, acc);
}

}  // namespace

// ------------------------------------------------------------------ launches
#define MR_ADJ_SC(FN, ...)                    \
  switch (g.scheme) {                         \
    case 0: FN<0><<<__VA_ARGS__; break;       \
    case 1: FN<1><<<__VA_ARGS__; break;       \
    case 2: FN<2><<<__VA_ARGS__; break;       \
    case 3: FN<3><<<__VA_ARGS__; break;       \
    case 4: FN<4><<<__VA_ARGS__; break;       \
  }

void mr_adj_collide(const Geo& g, const MeshDev& B, const double* z, double* lam, double* ds, int source,
                    double vol_J, cudaStream_t st, int grid) {
  MR_ADJ_SC(k_adj_collide, grid, 128, 0, st>>>(g, B, z, lam, ds, source, vol_J));
}
void mr_adj_transport(const Geo& g, const MeshDev& B, const double* W, const double* mu, double* aL, double* aI,
                      double* aG, cudaStream_t st, int grid) {
  MR_ADJ_SC(k_adj_transport, grid, 128, 0, st>>>(g, B, W, mu, aL, aI, aG));
}
void mr_adj_init(const Geo& g, const MeshDev& B, const double* cons, const double* lam, double* grad,
                 cudaStream_t st, int grid) {
  MR_ADJ_SC(k_adj_init, grid, 128, 0, st>>>(g, B, cons, lam, grad));
}
void mr_kinetic_energy(const Geo& g, const MeshDev& B, const double* LF, double vol_J, double* J, cudaStream_t st,
                       int grid) {
  MR_ADJ_SC(k_kinetic_energy, grid, 128, 0, st>>>(g, B, LF, vol_J, J));
}
void mr_adj_predict(const Geo& g, const MeshDev& B, int level, double* aL, double* aI, double* aG, cudaStream_t st,
                    int grid) {
  switch (g.d * 100 + g.Q) {
    case 102: k_adj_predict<1, 2><<<grid, 128, 0, st>>>(g, B, level, aL, aI, aG); break;
    case 103: k_adj_predict<1, 3><<<grid, 128, 0, st>>>(g, B, level, aL, aI, aG); break;
    case 209: k_adj_predict<2, 9><<<grid, 128, 0, st>>>(g, B, level, aL, aI, aG); break;
    case 216: k_adj_predict<2, 16><<<grid, 128, 0, st>>>(g, B, level, aL, aI, aG); break;
  }
}
void mr_adj_transfer(const Geo& g, const MeshDev& A, const MeshDev& B, const double* aLB, const double* aIB,
                     double* aLA, double* aIA, cudaStream_t st, int grid) {
  switch (g.Q) {
    case 2: k_adj_transfer<2><<<grid, 128, 0, st>>>(g, A, B, aLB, aIB, aLA, aIA); break;
    case 3: k_adj_transfer<3><<<grid, 128, 0, st>>>(g, A, B, aLB, aIB, aLA, aIA); break;
    case 9: k_adj_transfer<9><<<grid, 128, 0, st>>>(g, A, B, aLB, aIB, aLA, aIA); break;
    case 16: k_adj_transfer<16><<<grid, 128, 0, st>>>(g, A, B, aLB, aIB, aLA, aIA); break;
  }
}
void mr_adj_project(const Geo& g, const MeshDev& A, int level, double* aLA, double* aIA, cudaStream_t st, int grid) {
  switch (g.d * 100 + g.Q) {
    case 102: k_adj_project<1, 2><<<grid, 128, 0, st>>>(g, A, level, aLA, aIA); break;
    case 103: k_adj_project<1, 3><<<grid, 128, 0, st>>>(g, A, level, aLA, aIA); break;
    case 209: k_adj_project<2, 9><<<grid, 128, 0, st>>>(g, A, level, aLA, aIA); break;
    case 216: k_adj_project<2, 16><<<grid, 128, 0, st>>>(g, A, level, aLA, aIA); break;
  }
}

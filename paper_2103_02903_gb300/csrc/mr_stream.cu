// Data transfer to the new leaves (Sec. 5.1), reconstruction of the ghost
// cells, the leaf-reconstruction transport (Eq. AdaptiveAdvectionPhase,
// Eq. AdvectionOnBoundary) fused with the collision (Eq. AdaptiveCollision),
// and the input / output kernels of the C-ABI.
//
// Transport of a leaf (j, k) with a velocity along axis a.  Summed over the
// cells of the leaf that are transverse to a, the reconstruction of Sec. 4.4
// loses every term of the prediction operator that is odd in a transverse
// direction, so the incoming and outgoing sums of Eq. AdaptiveAdvectionPhase
// are 2^{(d-1)(J-j)} times the finest edge values of the one-dimensional
// reconstruction along a of the leaf's own row.  Those edge values are the
// flattened weights of Eq. PredictionWithMatrixNew applied to the five
// level-j values k-2..k+2 of the row (leaf values, projections of finer
// leaves, or predicted ghosts).  Where a neighbour k-1 or k+1 is refined,
// the details of its children (the critical case of Sec. 6.1) are added
// through the level-(j+1) weights; grading makes deeper corrections vanish.
#include "mr_common.cuh"

namespace {

// ------------------------------------------------------------------ schemes
template <int S>
struct Scheme;

// D1Q2: eta = (+1, -1), M = [[1, 1], [l, -l]], S = diag(0, s)
template <>
struct Scheme<0> {
  static constexpr int D = 1, Q = 2;
  __device__ static int axis(int p) { return 0; }
  __device__ static int sign(int p) { return p == 0 ? 1 : -1; }
  __device__ static int opp(int p) { return 1 - p; }
  __device__ static double meq1(const Geo& g, double m0) { return g.phys[0] * m0; }
  __device__ static void collide(const Geo& g, double* f) {
    const double L = g.lambda, s = g.s[0];
    const double m0 = f[0] + f[1];
    double m1 = L * (f[0] - f[1]);
    m1 = (1.0 - s) * m1 + s * meq1(g, m0);
    f[0] = 0.5 * (m0 + m1 / L);
    f[1] = 0.5 * (m0 - m1 / L);
  }
  __device__ static void equilibrium(const Geo& g, const double* u, double* f) {
    const double m1 = meq1(g, u[0]);
    f[0] = 0.5 * (u[0] + m1 / g.lambda);
    f[1] = 0.5 * (u[0] - m1 / g.lambda);
  }
};

// D1Q2 Burgers: m^eq_1 = u^2 / 2
template <>
struct Scheme<1> : Scheme<0> {
  __device__ static double meq1(const Geo&, double m0) { return 0.5 * m0 * m0; }
  __device__ static void collide(const Geo& g, double* f) {
    const double L = g.lambda, s = g.s[0];
    const double m0 = f[0] + f[1];
    double m1 = L * (f[0] - f[1]);
    m1 = (1.0 - s) * m1 + s * meq1(g, m0);
    f[0] = 0.5 * (m0 + m1 / L);
    f[1] = 0.5 * (m0 - m1 / L);
  }
  __device__ static void equilibrium(const Geo& g, const double* u, double* f) {
    const double m1 = meq1(g, u[0]);
    f[0] = 0.5 * (u[0] + m1 / g.lambda);
    f[1] = 0.5 * (u[0] - m1 / g.lambda);
  }
};

// D1Q3 shallow water: eta = (0, +1, -1), M = [[1,1,1],[0,l,-l],[0,l^2,l^2]]
template <>
struct Scheme<2> {
  static constexpr int D = 1, Q = 3;
  __device__ static int axis(int p) { return p == 0 ? -1 : 0; }
  __device__ static int sign(int p) { return p == 1 ? 1 : -1; }
  __device__ static int opp(int p) { return p == 0 ? 0 : 3 - p; }
  __device__ static void collide(const Geo& g, double* f) {
    const double L = g.lambda, s = g.s[0], gr = g.phys[0];
    const double m0 = f[0] + f[1] + f[2];
    const double m1 = L * (f[1] - f[2]);
    double m2 = L * L * (f[1] + f[2]);
    m2 = (1.0 - s) * m2 + s * (m1 * m1 / m0 + 0.5 * gr * m0 * m0);
    const double t = m2 / (L * L);
    f[0] = m0 - t;
    f[1] = 0.5 * (t + m1 / L);
    f[2] = 0.5 * (t - m1 / L);
  }
  __device__ static void equilibrium(const Geo& g, const double* u, double* f) {
    const double L = g.lambda;
    const double t = (u[1] * u[1] / u[0] + 0.5 * g.phys[0] * u[0] * u[0]) / (L * L);
    f[0] = u[0] - t;
    f[1] = 0.5 * (t + u[1] / L);
    f[2] = 0.5 * (t - u[1] / L);
  }
};

// D2Q4^4 Euler: per lattice i, eta = (1,0), (0,1), (-1,0), (0,-1)
template <>
struct Scheme<3> {
  static constexpr int D = 2, Q = 16;
  __device__ static int axis(int p) { return (p & 3) & 1; }
  __device__ static int sign(int p) { return (p & 3) < 2 ? 1 : -1; }
  __device__ static int opp(int p) { return (p & ~3) | ((p + 2) & 3); }
  __device__ static void fluxes(const Geo& g, const double* u, double* fx, double* fy) {
    const double rho = u[0], mx = u[1], my = u[2], E = u[3], gam = g.phys[0];
    const double irho = 1.0 / rho;  // one FP64 division per cell
    const double vx = mx * irho, vy = my * irho;
    const double pr = (gam - 1.0) * (E - 0.5 * (mx * vx + my * vy));
    fx[0] = mx; fx[1] = mx * vx + pr; fx[2] = my * vx; fx[3] = vx * (E + pr);
    fy[0] = my; fy[1] = mx * vy; fy[2] = my * vy + pr; fy[3] = vy * (E + pr);
  }
  __device__ static void from_moments(const Geo& g, double m0, double m1, double m2, double m3, double* f) {
    const double il = g.inv_lambda, il2 = il * il;
    const double a = 0.25 * m0, b = 0.5 * m1 * il, c = 0.5 * m2 * il, e = 0.25 * m3 * il2;
    f[0] = a + b + e;
    f[1] = a + c - e;
    f[2] = a - b + e;
    f[3] = a - c - e;
  }
  __device__ static void collide(const Geo& g, double* f) {
    const double L = g.lambda;
    double m[4][4], u[4], fx[4], fy[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double* fi = f + 4 * i;
      m[i][0] = fi[0] + fi[1] + fi[2] + fi[3];
      m[i][1] = L * (fi[0] - fi[2]);
      m[i][2] = L * (fi[1] - fi[3]);
      m[i][3] = L * L * (fi[0] - fi[1] + fi[2] - fi[3]);
      u[i] = m[i][0];
    }
    fluxes(g, u, fx, fy);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double sq = g.s[i], sxy = g.s[4 + i];
      const double m1 = (1.0 - sq) * m[i][1] + sq * fx[i];
      const double m2 = (1.0 - sq) * m[i][2] + sq * fy[i];
      const double m3 = (1.0 - sxy) * m[i][3];
      from_moments(g, m[i][0], m1, m2, m3, f + 4 * i);
    }
  }
  __device__ static void equilibrium(const Geo& g, const double* u, double* f) {
    double fx[4], fy[4];
    fluxes(g, u, fx, fy);
#pragma unroll
    for (int i = 0; i < 4; ++i) from_moments(g, u[i], fx[i], fy[i], 0.0, f + 4 * i);
  }
};

__device__ __forceinline__ double bc_value(int kind, const double* f, int p, int pd) {
  switch (kind) {
    case 1: return f[p];     // copy
    case 2: return f[pd];    // bounce back
    case 3: return -f[pd];   // anti bounce back
    default: return 0.0;
  }
}

// ------------------------------------------------------------------ transfer
// Thread layout of the transfer kernels: 32 cells (threadIdx.x) by up to 8
// populations (threadIdx.y), one population per warp.
template <int Q>
struct PopRows {
  static constexpr int value = Q < 8 ? Q : 8;
};

template <int Q>
__global__ void __launch_bounds__(256) k_remesh_copy(Geo g, MeshDev A, const double* __restrict__ LFold,
                                                     MeshDev B, double* LFnew) {
  constexpr int PY = PopRows<Q>::value;
  const int nL = B.cnt->total[MR_CLS_LEAF], nI = B.cnt->total[MR_CLS_INT];
  for (int t = blockIdx.x * 32 + threadIdx.x; t < nL + nI; t += gridDim.x * 32) {
    const bool leaf = t < nL;
    const int i = leaf ? t : t - nL;
    const int k = leaf ? MR_CLS_LEAF : MR_CLS_INT;
    const int l = B.lvl[k][i];
    const int32_t e = A.map[g.base[l] + B.code[k][i]];
    if (e != MR_MAP_NONE && (((uint32_t)e) >> 30) <= MR_CLS_INT) {
      const ValPtr s = mr_resolve(g, A, LFold, e);
      double* dst = leaf ? LFnew + i : B.IF + i;
      const size_t ds = leaf ? g.cap[0] : g.cap[1];
#pragma unroll
      for (int p = threadIdx.y; p < Q; p += PY) dst[(size_t)p * ds] = mr_ld(s, p);
      if (leaf && threadIdx.y == 0) B.src[i] = e;
    } else if (threadIdx.y == 0) {
      if (leaf)
        B.src[i] = -1;
      else
        mr_set_err(B.cnt, MR_DERR_INTERNAL);
    }
  }
}

// Ghosts and newly created leaves of one level: the prediction operator
// applied to level-1 values of the new mesh (all present by construction).
template <int D, int Q>
__global__ void __launch_bounds__(256) k_predict_level(Geo g, MeshDev B, double* LF, int level) {
  constexpr int PY = PopRows<Q>::value;
  const int gb = B.cnt->off[MR_CLS_GHOST][level], ge = B.cnt->off[MR_CLS_GHOST][level + 1];
  const int lb = B.cnt->off[MR_CLS_LEAF][level], le = B.cnt->off[MR_CLS_LEAF][level + 1];
  const int ng = ge - gb, total = ng + (le - lb);
  const double cs = (double)g.cross_sign;
  for (int t = blockIdx.x * 32 + threadIdx.x; t < total; t += gridDim.x * 32) {
    uint32_t code;
    double* out;
    size_t ostride;
    if (t < ng) {
      const int i = gb + t;
      code = B.code[MR_CLS_GHOST][i];
      out = B.GF + i;
      ostride = g.cap[2];
    } else {
      const int i = lb + (t - ng);
      if (B.src[i] >= 0) continue;
      code = B.code[MR_CLS_LEAF][i];
      out = LF + i;
      ostride = g.cap[0];
    }
    int px, py;
    mr_decode(g, level - 1, code >> D, px, py);
    int32_t st[9];
    if (!mr_stencil_entries<D>(g, B, level - 1, px, py, st)) {
      if (threadIdx.y == 0) mr_set_err(B.cnt, MR_DERR_INTERNAL);
      continue;
    }
    ValPtr sv[D == 2 ? 9 : 3];
#pragma unroll
    for (int k = 0; k < (D == 2 ? 9 : 3); ++k) sv[k] = mr_resolve(g, B, LF, st[k]);
    const int ci = (int)(code & ((1u << D) - 1u));
#pragma unroll
    for (int p = threadIdx.y; p < Q; p += PY) {
      double v[D == 2 ? 9 : 3];
#pragma unroll
      for (int k = 0; k < (D == 2 ? 9 : 3); ++k) v[k] = mr_ld(sv[k], p);
      out[(size_t)p * ostride] = mr_predict_fast<D>(v, ci, cs);
    }
  }
}

// ------------------------------------------------------------------ transport + collision
template <int S>
__global__ void __launch_bounds__(128) k_stream_collide(Geo g, MeshDev B, const double* __restrict__ LFin,
                                                        double* __restrict__ LFout,
                                                        const double* __restrict__ W, int do_stream,
                                                        int do_collide) {
  using Sc = Scheme<S>;
  constexpr int D = Sc::D, Q = Sc::Q;
  const int n = B.cnt->total[MR_CLS_LEAF];
  const double cs = (double)g.cross_sign;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int l = B.lvl[MR_CLS_LEAF][i];
    const uint32_t code = B.code[MR_CLS_LEAF][i];
    double f[Q], out[Q];
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      f[p] = __ldg(LFin + (size_t)p * g.cap[0] + i);
      out[p] = f[p];
    }
    if (do_stream) {
      int x, y;
      mr_decode(g, l, code, x, y);
      const double scale = ldexp(1.0, l - g.J);
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int k = a == 0 ? x : y;
        const int N = g.n[l][a];
        const int per = g.periodic[a];
        const int slot = mr_slot(k, N, per);
        const double* wP = W + MR_WIDX(l, a, slot, 0);
        const double* wM = W + MR_WIDX(l, a, slot, 1);
        // window: delta = -2, -1, +1, +2 along a
        ValPtr vp[4];
        bool has[4];
        int32_t ent[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int off = w < 2 ? w - 2 : w - 1;
          int nx = x + (a == 0 ? off : 0), ny = y + (a == 1 ? off : 0);
          has[w] = mr_nbr_mesh(g, l, nx, ny);
          ent[w] = has[w] ? B.map[g.base[l] + mr_encode(g, l, nx, ny)] : MR_MAP_NONE;
          if (has[w] && ent[w] == MR_MAP_NONE) {
            mr_set_err(B.cnt, MR_DERR_INTERNAL);
            has[w] = false;
          }
          vp[w] = mr_resolve(g, B, LFin, has[w] ? ent[w] : 0);
        }
#pragma unroll
        for (int p = 0; p < Q; ++p) {
          if (Sc::axis(p) != a) continue;
          const int sgn = Sc::sign(p);
          const double* w = sgn > 0 ? wP : wM;
          double acc = w[2] * f[p];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (has[q]) acc += w[q < 2 ? q : q + 1] * mr_ld(vp[q], p);
          if (!per) {
            if (sgn > 0 && k == 0) acc += bc_value(g.bc[2 * a], f, p, Sc::opp(p));
            if (sgn < 0 && k == N - 1) acc += bc_value(g.bc[2 * a + 1], f, p, Sc::opp(p));
          }
          out[p] += scale * acc;
        }
        // critical case: a refined neighbour on either side along a
#pragma unroll
        for (int side = -1; side <= 1; side += 2) {
          const int wi = side < 0 ? 1 : 2;
          if (!has[wi] || (((uint32_t)ent[wi]) >> 30) != MR_CLS_INT) continue;
          int nx = x + (a == 0 ? side : 0), ny = y + (a == 1 ? side : 0);
          mr_nbr_mesh(g, l, nx, ny);
          int32_t st[9];
          if (!mr_stencil_entries<D>(g, B, l, nx, ny, st)) {
            mr_set_err(B.cnt, MR_DERR_INTERNAL);
            continue;
          }
          ValPtr sv[D == 2 ? 9 : 3], cv[1 << D];
#pragma unroll
          for (int kk = 0; kk < (D == 2 ? 9 : 3); ++kk) sv[kk] = mr_resolve(g, B, LFin, st[kk]);
          const uint32_t ncode = mr_encode(g, l, nx, ny);
          bool ok = true;
#pragma unroll
          for (int ci = 0; ci < (1 << D); ++ci) {
            const int32_t e = B.map[g.base[l + 1] + ((ncode << D) | (uint32_t)ci)];
            ok = ok && e != MR_MAP_NONE;
            cv[ci] = mr_resolve(g, B, LFin, e);
          }
          if (!ok) {
            mr_set_err(B.cnt, MR_DERR_INTERNAL);
            continue;
          }
          const int N1 = g.n[l + 1][a];
#pragma unroll
          for (int p = 0; p < Q; ++p) {
            if (Sc::axis(p) != a) continue;
            const int sgn = Sc::sign(p);
            // the strip on the neighbour's side: incoming part if the
            // neighbour is upwind, outgoing part otherwise
            const bool incoming = (sgn > 0) == (side < 0);
            int c;  // child-level cell whose edge value is corrected
            if (sgn > 0)
              c = side < 0 ? 2 * k - 1 : 2 * k + 1;
            else
              c = side > 0 ? 2 * k + 2 : 2 * k;
            const int cslot = mr_slot(per ? 2 : c, N1, per);
            const double* wt = W + MR_WIDX(l + 1, a, cslot, sgn > 0 ? 2 : 3);
            double v[D == 2 ? 9 : 3];
#pragma unroll
            for (int kk = 0; kk < (D == 2 ? 9 : 3); ++kk) v[kk] = mr_ld(sv[kk], p);
            double corr = 0.0;
#pragma unroll
            for (int ci = 0; ci < (1 << D); ++ci) {
              const int sa = (ci >> a) & 1;
              const int delta = 2 * (k + side) + sa - c;
              if (delta < -2 || delta > 2) continue;
              const double det = mr_ld(cv[ci], p) - mr_predict_fast<D>(v, ci, cs);
              corr += wt[delta + 2] * det;
            }
            corr *= (D == 2 ? 0.5 : 1.0);
            out[p] += scale * (incoming ? corr : -corr);
          }
        }
      }
    }
    if (do_collide) Sc::collide(g, out);
    bool finite = true;
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      finite = finite && isfinite(out[p]);
      LFout[(size_t)p * g.cap[0] + i] = out[p];
    }
    if (!finite) mr_set_err(B.cnt, MR_DERR_NONFINITE);
  }
}

// ------------------------------------------------------------------ input / output
template <int S>
__global__ void __launch_bounds__(256) k_init_eq(Geo g, MeshDev B, const double* __restrict__ cons,
                                                 double* LF) {
  using Sc = Scheme<S>;
  const int n = B.cnt->total[MR_CLS_LEAF];
  const long long NJ = (long long)g.n[g.J][0] * (Sc::D == 2 ? g.n[g.J][1] : 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int x, y;
    mr_decode(g, g.J, B.code[MR_CLS_LEAF][i], x, y);
    const long long r = (long long)y * g.n[g.J][0] + x;
    double u[4], f[Sc::Q];
    for (int k = 0; k < g.ncons; ++k) u[k] = cons[k * NJ + r];
    Sc::equilibrium(g, u, f);
#pragma unroll
    for (int p = 0; p < Sc::Q; ++p) LF[(size_t)p * g.cap[0] + i] = f[p];
  }
}

__global__ void __launch_bounds__(256) k_gather_input(Geo g, MeshDev B, const int32_t* __restrict__ inidx,
                                                      long long nin, const double* __restrict__ fin,
                                                      double* LF) {
  const int n = B.cnt->total[MR_CLS_LEAF];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int l = B.lvl[MR_CLS_LEAF][i];
    const int32_t j = inidx[g.base[l] + B.code[MR_CLS_LEAF][i]];
    if (j < 0 || j >= nin) {
      mr_set_err(B.cnt, MR_DERR_INPUT);
      continue;
    }
    for (int p = 0; p < g.Q; ++p) LF[(size_t)p * g.cap[0] + i] = fin[(size_t)p * nin + j];
  }
}

__global__ void __launch_bounds__(256) k_leaves_out(Geo g, MeshDev B, const double* __restrict__ LF,
                                                    long long n, unsigned long long* keys,
                                                    signed char* levels, double* f) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (keys) keys[i] = B.code[MR_CLS_LEAF][i];
    if (levels) levels[i] = (signed char)B.lvl[MR_CLS_LEAF][i];
    if (f)
      for (int p = 0; p < g.Q; ++p) f[(size_t)p * n + i] = LF[(size_t)p * g.cap[0] + i];
  }
}

// Conserved moments on the uniform level `level`, row-major: values of the
// complete tree where present, the prediction of the level above otherwise.
template <int D>
__global__ void __launch_bounds__(256) k_project_dense(Geo g, MeshDev B, const double* __restrict__ LF,
                                                       int level, const double* __restrict__ prev,
                                                       double* cur) {
  const int nx = g.n[level][0], ny = D == 2 ? g.n[level][1] : 1;
  const long long N = (long long)nx * ny;
  const int pnx = level > g.Jmin ? g.n[level - 1][0] : 1;
  const long long PN = level > g.Jmin ? (long long)pnx * (D == 2 ? g.n[level - 1][1] : 1) : 1;
  const double cs = (double)g.cross_sign;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
       r += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(r % nx), y = (int)(r / nx);
    const int32_t e = B.map[g.base[level] + mr_encode(g, level, x, y)];
    if (e != MR_MAP_NONE && (((uint32_t)e) >> 30) <= MR_CLS_INT) {
      const ValPtr v = mr_resolve(g, B, LF, e);
      for (int k = 0; k < g.ncons; ++k) {
        double acc = 0.0;
        for (int p = 0; p < g.Q; ++p) acc += g.consw[k][p] * mr_ld(v, p);
        cur[k * N + r] = acc;
      }
    } else if (level > g.Jmin) {
      const int px = x >> 1, py = y >> 1;
      const int ci = (x & 1) | (D == 2 ? ((y & 1) << 1) : 0);
      for (int k = 0; k < g.ncons; ++k) {
        double v[9];
        for (int b = 0; b < (D == 2 ? 3 : 1); ++b)
          for (int a2 = 0; a2 < 3; ++a2) {
            int sx = px + a2 - 1, sy = D == 2 ? py + b - 1 : 0;
            mr_nbr_stencil(g, level - 1, sx, sy);
            v[b * 3 + a2] = prev[k * PN + (long long)sy * pnx + sx];
          }
        cur[k * N + r] = mr_predict_fast<D>(v, ci, cs);
      }
    } else {
      mr_set_err(B.cnt, MR_DERR_INTERNAL);
    }
  }
}

__global__ void k_count_updates(MeshCounts* cnt) {
  cnt->leaf_updates += cnt->total[MR_CLS_LEAF];
  cnt->steps += 1;
}

template <int Q>
void launch_remesh_t(const Geo& g, const MeshDev& A, const double* LFo, const MeshDev& B, double* LFn,
                     cudaStream_t st, int grid) {
  k_remesh_copy<Q><<<grid, dim3(32, PopRows<Q>::value), 0, st>>>(g, A, LFo, B, LFn);
}
template <int D, int Q>
void launch_predict_t(const Geo& g, const MeshDev& B, double* LF, int level, cudaStream_t st, int grid) {
  // `grid` is the maximum number of blocks; a block covers 32 cells
  const int need = (int)((2u * g.ncode[level] + 31) / 32);
  k_predict_level<D, Q><<<need < grid ? need : grid, dim3(32, PopRows<Q>::value), 0, st>>>(g, B, LF, level);
}

}  // namespace

void mr_launch_remesh_copy(const Geo& g, const MeshDev& A, const double* LF_old, const MeshDev& B,
                           double* LF_new, cudaStream_t st, int grid) {
  switch (g.Q) {
    case 2: launch_remesh_t<2>(g, A, LF_old, B, LF_new, st, grid); break;
    case 3: launch_remesh_t<3>(g, A, LF_old, B, LF_new, st, grid); break;
    case 9: launch_remesh_t<9>(g, A, LF_old, B, LF_new, st, grid); break;
    case 16: launch_remesh_t<16>(g, A, LF_old, B, LF_new, st, grid); break;
  }
}

void mr_launch_predict_level(const Geo& g, const MeshDev& B, double* LF, int level, cudaStream_t st,
                             int grid) {
  switch (g.d * 100 + g.Q) {
    case 102: launch_predict_t<1, 2>(g, B, LF, level, st, grid); break;
    case 103: launch_predict_t<1, 3>(g, B, LF, level, st, grid); break;
    case 216: launch_predict_t<2, 16>(g, B, LF, level, st, grid); break;
    case 209: launch_predict_t<2, 9>(g, B, LF, level, st, grid); break;
  }
}

void mr_launch_stream_collide(const Geo& g, const MeshDev& B, const double* LF_in, double* LF_out,
                              const double* W, int do_stream, int do_collide, cudaStream_t st,
                              int grid) {
  switch (g.scheme) {
    case 0: k_stream_collide<0><<<grid, 128, 0, st>>>(g, B, LF_in, LF_out, W, do_stream, do_collide); break;
    case 1: k_stream_collide<1><<<grid, 128, 0, st>>>(g, B, LF_in, LF_out, W, do_stream, do_collide); break;
    case 2: k_stream_collide<2><<<grid, 128, 0, st>>>(g, B, LF_in, LF_out, W, do_stream, do_collide); break;
    case 3: k_stream_collide<3><<<grid, 128, 0, st>>>(g, B, LF_in, LF_out, W, do_stream, do_collide); break;
  }
}

void mr_launch_init_eq(const Geo& g, const MeshDev& B, const double* cons, double* LF, cudaStream_t st,
                       int grid) {
  switch (g.scheme) {
    case 0: k_init_eq<0><<<grid, 256, 0, st>>>(g, B, cons, LF); break;
    case 1: k_init_eq<1><<<grid, 256, 0, st>>>(g, B, cons, LF); break;
    case 2: k_init_eq<2><<<grid, 256, 0, st>>>(g, B, cons, LF); break;
    case 3: k_init_eq<3><<<grid, 256, 0, st>>>(g, B, cons, LF); break;
  }
}

void mr_launch_gather_input(const Geo& g, const MeshDev& B, const int32_t* inidx, long long n,
                            const double* fin, double* LF, cudaStream_t st, int grid) {
  k_gather_input<<<grid, 256, 0, st>>>(g, B, inidx, n, fin, LF);
}

void mr_launch_leaves_out(const Geo& g, const MeshDev& B, const double* LF, long long n,
                          unsigned long long* keys, signed char* levels, double* f, cudaStream_t st,
                          int grid) {
  k_leaves_out<<<grid, 256, 0, st>>>(g, B, LF, n, keys, levels, f);
}

void mr_launch_project_dense(const Geo& g, const MeshDev& B, const double* LF, int level,
                             const double* prev, double* cur, cudaStream_t st, int grid) {
  if (g.d == 1)
    k_project_dense<1><<<grid, 256, 0, st>>>(g, B, LF, level, prev, cur);
  else
    k_project_dense<2><<<grid, 256, 0, st>>>(g, B, LF, level, prev, cur);
}

void mr_launch_count_updates(MeshCounts* cnt, cudaStream_t st) { k_count_updates<<<1, 1, 0, st>>>(cnt); }

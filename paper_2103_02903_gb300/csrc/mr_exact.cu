// The "original adaptive" collision (Sec. 5.3, the right-hand side of
// Eq. sourceoferror): instead of colliding each leaf's averages
// (Eq. AdaptiveCollision), the post-transport data are reconstructed on every
// finest cell, each finest cell is collided, and every leaf receives the
// average of its finest cells B_{j,k} (Eq. CellSplitting).
//
// The reconstruction is dense, level by level, in one FP64 buffer
// [Q][cells of levels J_min..J] indexed like the dense per-level map:
//   up   (J .. J_min): a leaf takes its post-transport value, an internal
//        cell the average of its children (Def. Projection, children in
//        index order, then 2^-d);
//   down (J_min+1 .. J): every cell outside the tree takes the prediction
//        of half-width s from its parent's (2s+1)^d stencil (the
//        reconstruction operator of Sec. 4.4); on level J every cell is
//        then collided in place;
//   average (J-1 .. J_min): every cell outside the tree, and every leaf,
//        takes the average of its children (collided on level J, averaged
//        below): the leaf's average over its finest cells, 2^{-d(J-j)} times
//        their sum, formed level by level so that no thread sums a large
//        leaf alone; then each leaf takes its cell's value and the obstacle
//        penalisation follows as after the leaf collision.
// Single instances in the FP64 form; the cost is that of the dense level-J
// grid, the explosion the paper warns about, which 2D grids up to J = 10 fit.
#include "mr_wide.cuh"

namespace {

template <int D>
__global__ void __launch_bounds__(256) k_exact_up(const InstDev* __restrict__ IB, int dst, int kl,
                                                  double* __restrict__ Fd, long long nd) {
  __shared__ InstDev si;
  int have = -1;
  mr_inst_use(si, have, IB, 0);
  mr_grid_dep();
  const Geo& g = si.g;
  const MeshDev& B = si.mesh[dst];
  const int l = g.Jmin + kl;
  const double* LF = (const double*)si.fstate;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncode[l]) return;
  const uint32_t gi = g.base[l] + c;
  const int32_t e = B.map[gi];
  if (e == MR_MAP_NONE) return;
  const uint32_t cls = ((uint32_t)e) >> 30, idx = (uint32_t)e & 0x3FFFFFFFu;
  if (cls == MR_CLS_LEAF) {
    for (int p = 0; p < g.Q; ++p) Fd[(size_t)p * nd + gi] = LF[(size_t)p * g.cap[0] + idx];
  } else if (cls == MR_CLS_INT) {
    const double scale = D == 1 ? 0.5 : D == 2 ? 0.25 : 0.125;  // 2^-d
    const uint32_t cb = g.base[l + 1] + (c << D);
    for (int p = 0; p < g.Q; ++p) {
      double acc = 0.0;
#pragma unroll
      for (int ci = 0; ci < (1 << D); ++ci) acc = __dadd_rn(acc, Fd[(size_t)p * nd + cb + ci]);
      Fd[(size_t)p * nd + gi] = __dmul_rn(acc, scale);
    }
  }
}

template <int SC>
__global__ void __launch_bounds__(256) k_exact_down(const InstDev* __restrict__ IB, int dst, int kl,
                                                    double* __restrict__ Fd, long long nd) {
  using Sc = Scheme<SC>;
  constexpr int D = Sc::D, Q = Sc::Q, NS = D == 2 ? 9 : 3;
  __shared__ InstDev si;
  int have = -1;
  mr_inst_use(si, have, IB, 0);
  mr_grid_dep();
  const Geo& g = si.g;
  const MeshDev& B = si.mesh[dst];
  const int l = g.Jmin + kl;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncode[l]) return;
  const uint32_t gi = g.base[l] + c;
  const int32_t e = B.map[gi];
  const bool tree = e != MR_MAP_NONE && (((uint32_t)e) >> 30) <= MR_CLS_INT;
  double f[Q];
  if (tree) {
    if (l < g.J) return;  // set on the way up
#pragma unroll
    for (int p = 0; p < Q; ++p) f[p] = Fd[(size_t)p * nd + gi];
  } else {
    int x, y;
    mr_decode(g, l, c, x, y);
    uint32_t st[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      int sx = (x >> 1) + (k % 3) - 1, sy = D == 2 ? (y >> 1) + (k / 3) - 1 : 0;
      mr_nbr_stencil(g, l - 1, sx, sy);
      st[k] = g.base[l - 1] + mr_encode(g, l - 1, sx, sy);
    }
    const int ci = (x & 1) | (D == 2 ? (y & 1) << 1 : 0);
    const double cs = g.cross_sign;
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      double v[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) v[k] = Fd[(size_t)p * nd + st[k]];
      f[p] = predict_c<D, double>(v, ci, cs);
    }
  }
  if (l == g.J) Sc::template collide<double>(g, f);
#pragma unroll
  for (int p = 0; p < Q; ++p) Fd[(size_t)p * nd + gi] = f[p];
}

// The same for the prediction of half-width s = 2, 3.
template <int SC, int S>
__global__ void __launch_bounds__(256) k_exact_down_w(const InstDev* __restrict__ IB, int dst, int kl,
                                                      double* __restrict__ Fd, long long nd) {
  using Sc = Scheme<SC>;
  using B = WBox<Sc::D, S>;
  constexpr int D = Sc::D, Q = Sc::Q;
  __shared__ InstDev si;
  int have = -1;
  mr_inst_use(si, have, IB, 0);
  mr_grid_dep();
  const Geo& g = si.g;
  const MeshDev& Bm = si.mesh[dst];
  const int l = g.Jmin + kl;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncode[l]) return;
  const uint32_t gi = g.base[l] + c;
  const int32_t e = Bm.map[gi];
  const bool tree = e != MR_MAP_NONE && (((uint32_t)e) >> 30) <= MR_CLS_INT;
  double f[Q];
  if (tree) {
    if (l < g.J) return;  // set on the way up
    for (int p = 0; p < Q; ++p) f[p] = Fd[(size_t)p * nd + gi];
  } else {
    int x[3] = {0, 0, 0};
    mr_decode_d<D>(g, l, c, x);
    uint32_t st[B::N];
    for (int k = 0; k < B::N; ++k) {
      int s[3] = {(x[0] >> 1) + k % B::W1 - S, D >= 2 ? (x[1] >> 1) + (k / B::W1) % B::W1 - S : 0, 0};
      mr_nbr_stencil_d<D>(g, l - 1, s);
      st[k] = g.base[l - 1] + mr_encode_d<D>(g, l - 1, s);
    }
    const int ci = (x[0] & 1) | (D == 2 ? (x[1] & 1) << 1 : 0);
    for (int p = 0; p < Q; ++p) {
      double v[B::N];
      for (int k = 0; k < B::N; ++k) v[k] = Fd[(size_t)p * nd + st[k]];
      f[p] = wide_predict<D, S, double, false>(v, ci, g.cross_sign);
    }
  }
  if (l == g.J) Sc::template collide<double>(g, f);
  for (int p = 0; p < Q; ++p) Fd[(size_t)p * nd + gi] = f[p];
}

template <int D>
__global__ void __launch_bounds__(256) k_exact_average(const InstDev* __restrict__ IB, int dst, int kl,
                                                       double* __restrict__ Fd, long long nd) {
  __shared__ InstDev si;
  int have = -1;
  mr_inst_use(si, have, IB, 0);
  mr_grid_dep();
  const Geo& g = si.g;
  const MeshDev& B = si.mesh[dst];
  const int l = g.Jmin + kl;
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncode[l]) return;
  const uint32_t gi = g.base[l] + c;
  const int32_t e = B.map[gi];
  if (e != MR_MAP_NONE && (((uint32_t)e) >> 30) == MR_CLS_INT) return;  // not inside a leaf
  const double scale = D == 1 ? 0.5 : D == 2 ? 0.25 : 0.125;  // 2^-d
  const uint32_t cb = g.base[l + 1] + (c << D);
  for (int p = 0; p < g.Q; ++p) {
    double acc = 0.0;
#pragma unroll
    for (int ci = 0; ci < (1 << D); ++ci) acc += Fd[(size_t)p * nd + cb + ci];
    Fd[(size_t)p * nd + gi] = acc * scale;
  }
}

template <int SC>
__global__ void __launch_bounds__(128) k_exact_leaves(const InstDev* __restrict__ IB, int dst,
                                                      const double* __restrict__ Fd, long long nd) {
  using Sc = Scheme<SC>;
  constexpr int Q = Sc::Q;
  __shared__ InstDev si;
  int have = -1;
  mr_inst_use(si, have, IB, 0);
  mr_grid_dep();
  const Geo& g = si.g;
  const MeshDev& B = si.mesh[dst];
  double* LF = (double*)si.fstate;
  const int n = B.cnt->total[MR_CLS_LEAF];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int l = B.lvl[MR_CLS_LEAF][i];
    const uint32_t code = B.code[MR_CLS_LEAF][i];
    const uint32_t gi = g.base[l] + code;
    double f[Q];
#pragma unroll
    for (int p = 0; p < Q; ++p) f[p] = Fd[(size_t)p * nd + gi];
    if constexpr (Sc::DIAG) {
      if (g.obstacle) {
        const double phi = obstacle_fraction(g, l, code);
        if (phi > 0.0) {
#pragma unroll
          for (int p = 0; p < Q; ++p) f[p] = phi * g.feq0[p] + (1.0 - phi) * f[p];
        }
      }
    }
    bool finite = true;
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      finite = finite && is_finite_bits(f[p]);
      LF[(size_t)p * g.cap[0] + i] = f[p];
    }
    if (!finite) mr_set_err(B.cnt, MR_DERR_NONFINITE);
  }
}

template <int SC>
void launch_exact_t(const Group& G, int dst, double* Fd, long long nd, cudaStream_t st) {
  constexpr int D = Scheme<SC>::D;
  const int span = G.span;
  auto cells = [&](int k) { return k == 0 ? G.proj_cells[span] : G.pred_cells[k]; };  // level J_min + k
  for (int k = span; k >= 0; --k)
    mr_launch_pdl(k_exact_up<D>, (unsigned)((cells(k) + 255) / 256), 256, 0, st, G.dev, dst, k, Fd, nd);
  for (int k = 1; k <= span; ++k) {
    const unsigned grid = (unsigned)((cells(k) + 255) / 256);
    if (G.s == 2)
      mr_launch_pdl(k_exact_down_w<SC, 2>, grid, 256, 0, st, G.dev, dst, k, Fd, nd);
    else if (G.s == 3)
      mr_launch_pdl(k_exact_down_w<SC, 3>, grid, 256, 0, st, G.dev, dst, k, Fd, nd);
    else
      mr_launch_pdl(k_exact_down<SC>, grid, 256, 0, st, G.dev, dst, k, Fd, nd);
  }
  for (int k = span - 1; k >= 0; --k)
    mr_launch_pdl(k_exact_average<D>, (unsigned)((cells(k) + 255) / 256), 256, 0, st, G.dev, dst, k, Fd, nd);
  mr_launch_pdl(k_exact_leaves<SC>, (unsigned)(G.nsm * 8), 128, 0, st, G.dev, dst, (const double*)Fd, nd);
}

}  // namespace

int mr_launch_exact_collision(const Group& G, int dst, double* Fd, long long nd, cudaStream_t st) {
  switch (G.scheme) {
    case 0: launch_exact_t<0>(G, dst, Fd, nd, st); break;
    case 1: launch_exact_t<1>(G, dst, Fd, nd, st); break;
    case 2: launch_exact_t<2>(G, dst, Fd, nd, st); break;
    case 3: launch_exact_t<3>(G, dst, Fd, nd, st); break;
    case 4: launch_exact_t<4>(G, dst, Fd, nd, st); break;
    default: return 0;
  }
  return 3 * G.span + 2;
}

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
//
// Every kernel is instantiated per storage / compute form (FormT): values
// are stored as FormT::S and transported / collided in FormT::C.  The
// transfer and the ghost prediction are linear and exact on constants and
// act on stored values; transport, collision and input / output add the
// offset of the 16-bit forms back.
#include "mr_schemes.cuh"

namespace {

// ------------------------------------------------------------------ transfer
// Thread layout of the transfer kernels: 32 cells (threadIdx.x) by up to 8
// populations (threadIdx.y), one population per warp.
template <int Q, int F>
__global__ void __launch_bounds__(256) k_remesh_copy(const InstDev* __restrict__ IB, int ngrp, int cur) {
  using S = typename FormT<F>::S;
  constexpr int PY = PopRows<Q>::value;
  extern __shared__ int pre[];
  __shared__ InstDev si;
  int have = -1;
  mr_inst_prefetch(si, have, IB, ngrp);
  mr_grid_dep();  // after the copy of the descriptor, which no step kernel writes
  const int tiles = mr_group_prefix(pre, ngrp, [&](int b) {
    const MeshCounts* c = IB[b].mesh[1 - cur].cnt;
    return (c->total[MR_CLS_LEAF] + c->total[MR_CLS_INT] + 31) / 32;
  });
  for (int tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
    const int b = mr_group_find(pre, ngrp, tt);
    mr_inst_use(si, have, IB, b);
    const Geo& g = si.g;
    const MeshDev& A = si.mesh[cur];
    const MeshDev& B = si.mesh[1 - cur];
    const void* LFold = si.fstate;
    void* LFnew = si.fscratch;
    const int nL = B.cnt->total[MR_CLS_LEAF], nI = B.cnt->total[MR_CLS_INT];
    const int t = (tt - pre[b]) * 32 + threadIdx.x;
    if (t >= nL + nI) continue;
    const bool leaf = t < nL;
    const int i = leaf ? t : t - nL;
    const int k = leaf ? MR_CLS_LEAF : MR_CLS_INT;
    const int l = B.lvl[k][i];
    const int32_t e = A.map[g.base[l] + B.code[k][i]];
    if (e != MR_MAP_NONE && (((uint32_t)e) >> 30) <= MR_CLS_INT) {
      const ValPtr<S> s = mr_resolve<S>(g, A, LFold, e);
      S* dst = leaf ? (S*)LFnew + i : (S*)B.IF + i;
      const size_t ds = leaf ? g.cap[0] : g.cap[1];
#pragma unroll
      for (int p = threadIdx.y; p < Q; p += PY) dst[(size_t)p * ds] = __ldg(s.p + (size_t)p * s.stride);
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
// 2D and 1D: at most 64 registers, 4 blocks per SM; 3D: 2 blocks, 128
// registers
template <int D, int Q, int F>
__global__ void __launch_bounds__(256, D == 3 ? 2 : 4) k_predict_level(const InstDev* __restrict__ IB, int ngrp, int dst,
                                                                       int kl) {
  using S = typename FormT<F>::S;
  using C = typename FormT<F>::C;
  constexpr int PY = PopRows<Q>::value;
  extern __shared__ int pre[];
  __shared__ InstDev si;
  int have = -1;
  mr_inst_prefetch(si, have, IB, ngrp);
  mr_grid_dep();  // after the copy of the descriptor, which no step kernel writes
  const int tiles = mr_group_prefix(pre, ngrp, [&](int b) {
    const Geo& gb = IB[b].g;
    const int l = gb.Jmin + kl;
    if (l > gb.J) return 0;
    const MeshCounts* c = IB[b].mesh[dst].cnt;
    return (c->off[MR_CLS_GHOST][l + 1] - c->off[MR_CLS_GHOST][l] + c->off[MR_CLS_LEAF][l + 1] -
            c->off[MR_CLS_LEAF][l] + 31) / 32;
  });
  // the parent's 3^D stencil entries, looked up once per cell (spread over
  // the population rows) and shared through the block
  constexpr int NS = Pow3<D>::value;
  __shared__ int32_t sent[NS][32];
  for (int tt = blockIdx.x; tt < tiles; tt += gridDim.x) {  // uniform over the block
    const int b = mr_group_find(pre, ngrp, tt);
    mr_inst_use(si, have, IB, b);
    const Geo& g = si.g;
    const MeshDev& B = si.mesh[dst];
    void* LF = si.fscratch;
    const int level = g.Jmin + kl;
    const int gb = B.cnt->off[MR_CLS_GHOST][level], ge = B.cnt->off[MR_CLS_GHOST][level + 1];
    const int lb = B.cnt->off[MR_CLS_LEAF][level], le = B.cnt->off[MR_CLS_LEAF][level + 1];
    const int ng = ge - gb, total = ng + (le - lb);
    const C cs = MR_K(C, g, cross_sign);
    const int t = (tt - pre[b]) * 32 + threadIdx.x;
    bool active = t < total;
    uint32_t code = 0;
    S* out = nullptr;
    size_t ostride = 0;
    if (active) {
      if (t < ng) {
        const int i = gb + t;
        code = B.code[MR_CLS_GHOST][i];
        out = (S*)B.GF + i;
        ostride = g.cap[2];
      } else {
        const int i = lb + (t - ng);
        active = B.src[i] < 0;  // a leaf carried over keeps its transferred values
        code = B.code[MR_CLS_LEAF][i];
        out = (S*)LF + i;
        ostride = g.cap[0];
      }
    }
    __syncthreads();  // the previous tile's readers of sent are done
    if (active) {
      int pc[3] = {0, 0, 0};
      mr_decode_d<D>(g, level - 1, code >> D, pc);
      for (int e = threadIdx.y; e < NS; e += PY) sent[e][threadIdx.x] = mr_stencil_entry_d<D>(g, B, level - 1, pc, e);
    }
    __syncthreads();
    if (!active) continue;
    ValPtr<S> sv[NS];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const int32_t e = sent[k][threadIdx.x];
      ok = ok && e != MR_MAP_NONE;
      sv[k] = mr_resolve<S>(g, B, LF, e);
    }
    if (!ok) {
      if (threadIdx.y == 0) mr_set_err(B.cnt, MR_DERR_INTERNAL);
      continue;
    }
    const int ci = (int)(code & ((1u << D) - 1u));
#pragma unroll
    for (int p = threadIdx.y; p < Q; p += PY) {
      C v[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) v[k] = ld_c<C>(sv[k], p);
      out[(size_t)p * ostride] = mr_from_d<S>((double)predict_c<D, C>(v, ci, cs));
    }
  }
}

// ------------------------------------------------------------------ axis strips
// The parts of the transport that few leaves take (a non-periodic face, a
// refined neighbour) loop over the populations at run time and leave their
// terms in a per-thread shared-memory buffer `tmp`; the caller adds them to
// the register accumulators at the same point of the sum as an inline term
// would be.  One short loop body instead of one copy per population keeps
// the kernel's code small enough for the instruction cache.
#define MR_WIN_TPB 128  // threads per block of the transport kernel

// stride of the per-thread shared buffers: odd, so that 32 threads (or 16
// for 8-byte values) hit distinct banks
template <int Q>
struct ThreadStride {
  static constexpr int value = Q | 1;
};

// Boundary values of the populations entering through the face crossed
// upwind along a (lo: the face before cell 0, hi: the one after N-1).
template <class Sc, class C>
__device__ __forceinline__ void bc_terms(const Geo& g, int a, bool lo, bool hi, const C* fs, C* tmp) {
#pragma unroll 1
  for (int p = 0; p < Sc::Q; ++p) {
    const int sgn = eta_of<Sc>(p, a);
    if (sgn > 0 && lo)
      tmp[p] = bc_value<C>(g, g.bc[2 * a], fs, p, Sc::opp(p));
    else if (sgn < 0 && hi)
      tmp[p] = bc_value<C>(g, g.bc[2 * a + 1], fs, p, Sc::opp(p));
  }
}

// Critical case (Sec. 6.1) along axis a: the neighbour on `side` is
// refined, so the finest value at the shared edge is its children's, not
// the prediction from level l.  tmp[p] = the term to add for population p
// (scaled): the edge cell's detail through the level-(l+1) edge weights,
// with the sign of the strip part (incoming if the neighbour is upwind).
template <class Sc, int F>
__device__ __forceinline__ void crit_axis_terms(const Geo& g, const typename FormT<F>::C* __restrict__ W, int l,
                                                int a, int k, int side, int per,
                                                const ValPtr<typename FormT<F>::S>* sv,
                                                const ValPtr<typename FormT<F>::S>* cv, typename FormT<F>::C scale,
                                                typename FormT<F>::C* tmp) {
  using C = typename FormT<F>::C;
  constexpr int D = Sc::D, NS = Pow3<D>::value;
  const C cs = MR_K(C, g, cross_sign);
  const int N1 = g.n[l + 1][a];
#pragma unroll 1
  for (int p = 0; p < Sc::Q; ++p) {
    const int sgn = eta_of<Sc>(p, a);
    if (sgn == 0) continue;
    const bool incoming = (sgn > 0) == (side < 0);
    int c;  // child-level cell whose edge value is corrected
    if (sgn > 0)
      c = side < 0 ? 2 * k - 1 : 2 * k + 1;
    else
      c = side > 0 ? 2 * k + 2 : 2 * k;
    const int cslot = mr_slot(per ? 2 : c, N1, per);
    const C* wt = W + MR_WIDX(l + 1, a, cslot, sgn > 0 ? 2 : 3);
    // details are exact on constants: stored values suffice
    C v[NS];
#pragma unroll
    for (int kk = 0; kk < NS; ++kk) v[kk] = ld_c<C>(sv[kk], p);
    C corr = (C)0;
#pragma unroll
    for (int ci = 0; ci < (1 << D); ++ci) {
      const int sa = (ci >> a) & 1;
      const int delta = 2 * (k + side) + sa - c;
      if (delta < -2 || delta > 2) continue;
      const C det = ld_c<C>(cv[ci], p) - predict_c<D, C>(v, ci, cs);
      corr += wt[delta + 2] * det;
    }
    corr *= (C)1 / (C)(1 << (D - 1));  // average over the 2^{d-1} children on the shared face
    tmp[p] = scale * (incoming ? corr : -corr);
  }
}

// The same terms from the children's details computed once per refined cell
// (k_edge_details; D2Q9): det[(child * Q + p) * cap_int + ridx].
template <class Sc, int F>
__device__ __forceinline__ void crit_axis_terms_det(const Geo& g, const typename FormT<F>::C* __restrict__ W,
                                                    const typename FormT<F>::C* __restrict__ det, int l, int a, int k,
                                                    int side, int per, uint32_t ridx, typename FormT<F>::C scale,
                                                    typename FormT<F>::C* tmp) {
  using C = typename FormT<F>::C;
  constexpr int D = Sc::D;
  const int N1 = g.n[l + 1][a];
  const size_t cap1 = g.cap[1];
#pragma unroll 1
  for (int p = 0; p < Sc::Q; ++p) {
    const int sgn = eta_of<Sc>(p, a);
    if (sgn == 0) continue;
    const bool incoming = (sgn > 0) == (side < 0);
    int c;  // child-level cell whose edge value is corrected
    if (sgn > 0)
      c = side < 0 ? 2 * k - 1 : 2 * k + 1;
    else
      c = side > 0 ? 2 * k + 2 : 2 * k;
    const int cslot = mr_slot(per ? 2 : c, N1, per);
    const C* wt = W + MR_WIDX(l + 1, a, cslot, sgn > 0 ? 2 : 3);
    C corr = (C)0;
#pragma unroll
    for (int ci = 0; ci < (1 << D); ++ci) {
      const int sa = (ci >> a) & 1;
      const int delta = 2 * (k + side) + sa - c;
      if (delta < -2 || delta > 2) continue;
      corr += wt[delta + 2] * det[((size_t)ci * Sc::Q + p) * cap1 + ridx];
    }
    corr *= (C)1 / (C)(1 << (D - 1));  // average over the 2^{d-1} children on the shared face
    tmp[p] = scale * (incoming ? corr : -corr);
  }
}

__device__ __forceinline__ bool win_stencil(const Geo& g, int l, int x, int y, int ox, int oy,
                                            const int32_t (*win)[MR_WIN_TPB], int32_t* st);

// Strip term of axis a for every population moving along a: the flattened
// weights of the leaf's slot applied to the level-l window (cells -2, -1,
// +1, +2 in vp, present where has), the boundary values of a non-periodic
// face, and the critical-case corrections of a refined neighbour on either
// side.  The neighbour's prediction stencil comes from the 5 x 5 block in
// shared memory (win) when there is one, from the index map otherwise.
template <class Sc, int F>
__device__ __forceinline__ void stream_axis(const Geo& g, const MeshDev& B,
                                            const typename FormT<F>::S* __restrict__ LFin,
                                            const typename FormT<F>::C* __restrict__ W, int l, int a, int x, int y,
                                            int z, const ValPtr<typename FormT<F>::S>* vp, const bool* has,
                                            const int32_t* ent, const typename FormT<F>::C* fs,
                                            const typename FormT<F>::C* offv, typename FormT<F>::C* out,
                                            typename FormT<F>::C scale, typename FormT<F>::C* tmp,
                                            const int32_t (*win)[MR_WIN_TPB],
                                            const typename FormT<F>::C* __restrict__ det = nullptr) {
  using S = typename FormT<F>::S;
  using C = typename FormT<F>::C;
  constexpr int D = Sc::D, Q = Sc::Q, NS = Pow3<D>::value;
  const int k = a == 0 ? x : (a == 1 ? y : z);
  const int N = g.n[l][a];
  const int per = g.periodic[a];
  const int slot = mr_slot(k, N, per);
  const C* wP = W + MR_WIDX(l, a, slot, 0);
  const C* wM = W + MR_WIDX(l, a, slot, 1);
  const bool lo = !per && k == 0, hi = !per && k == N - 1;
  if (lo || hi) bc_terms<Sc, C>(g, a, lo, hi, fs, tmp);
#pragma unroll
  for (int p = 0; p < Q; ++p) {
    const int sgn = eta_of<Sc>(p, a);
    if (sgn == 0) continue;
    const C* w = sgn > 0 ? wP : wM;
    C acc = w[2] * fs[p];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (has[q]) acc += w[q < 2 ? q : q + 1] * ld_off<F>(vp[q], p, offv);
    if (sgn > 0 && lo) acc += tmp[p];
    if (sgn < 0 && hi) acc += tmp[p];
    out[p] += scale * acc;
  }
  // refined neighbours at -1 (bit 0) and +1 (bit 1); one rolled loop over them
  const uint32_t refined = (has[1] && (((uint32_t)ent[1]) >> 30) == MR_CLS_INT ? 1u : 0u) |
                           (has[2] && (((uint32_t)ent[2]) >> 30) == MR_CLS_INT ? 2u : 0u);
#pragma unroll 1
  for (int si = 0; si < 2; ++si) {
    if (!((refined >> si) & 1u)) continue;
    const int side = si == 0 ? -1 : 1;
    if constexpr (Sc::DIAG) {  // the details were computed once per refined cell
      crit_axis_terms_det<Sc, F>(g, W, det, l, a, k, side, per, (uint32_t)ent[si == 0 ? 1 : 2] & 0x3FFFFFFFu, scale,
                                 tmp);
#pragma unroll
      for (int p = 0; p < Q; ++p)
        if (eta_of<Sc>(p, a) != 0) out[p] += tmp[p];
      continue;
    }
    const int ox = a == 0 ? side : 0, oy = a == 1 ? side : 0;
    int nb[3] = {x, y, z};
    nb[a] += side;
    mr_nbr_mesh_d<D>(g, l, nb);
    int32_t st[NS];
    bool ok;
    if constexpr (D == 2)
      ok = win ? win_stencil(g, l, x, y, ox, oy, win, st) : mr_stencil_entries_d<D>(g, B, l, nb, st);
    else
      ok = mr_stencil_entries_d<D>(g, B, l, nb, st);
    const uint32_t ncode = mr_encode_d<D>(g, l, nb);
    ValPtr<S> sv[NS], cv[1 << D];
#pragma unroll
    for (int ci = 0; ci < (1 << D); ++ci) {
      const int32_t e = B.map[g.base[l + 1] + ((ncode << D) | (uint32_t)ci)];
      ok = ok && e != MR_MAP_NONE;
      cv[ci] = mr_resolve<S>(g, B, LFin, e);
    }
    if (!ok) {
      mr_set_err(B.cnt, MR_DERR_INTERNAL);
      continue;
    }
#pragma unroll
    for (int kk = 0; kk < NS; ++kk) sv[kk] = mr_resolve<S>(g, B, LFin, st[kk]);
    crit_axis_terms<Sc, F>(g, W, l, a, k, side, per, sv, cv, scale, tmp);
#pragma unroll
    for (int p = 0; p < Q; ++p)
      if (eta_of<Sc>(p, a) != 0) out[p] += tmp[p];
  }
}

// ------------------------------------------------------------------ diagonal velocities
// Transport of a leaf of a lattice with diagonal velocities (D2Q9).
//
// Every cell the leaf reads lies in the 5 x 5 block of level-l cells around
// it: the flattened windows of both axes, the four single finest cells of
// each diagonal velocity, and the prediction stencil of any refined cell
// among the 8 neighbours.  The block's 24 map entries are looked up once,
// all loads issued together, and kept in shared memory, so that every later
// read of an entry is a shared-memory load instead of a dependent global
// one.
//
// Diagonal velocities eta = (sx, sy) (Eq. AdaptiveAdvectionPhase).  The sum
// over E minus the sum over A is the strip term of each axis, evaluated as
// for an axis velocity, plus four single finest cells at the ends of the
// strips: + the cell diagonally upwind of the leaf, + the leaf's own
// downwind corner cell, - the two cells that mix the two.  With the
// tensor-product prediction a finest value is the product of the
// one-dimensional reconstructions, so the four cells are the product of the
// two axes' in-minus-out flattened weights applied to the block of level-l
// values.  A refined cell among the 8 neighbours adds the details of its
// children through the level-(l+1) edge weights (the critical case of Sec.
// 6.1; grading keeps deeper levels away).  At a corner of a non-periodic
// domain the outside cells take the boundary value of the face crossed first
// along x, so after the two strips the four cells leave minus the value of
// the y face.
#define MR_WIN_OUT ((int32_t)0xC0000000)  // block cell outside a non-periodic domain

__device__ __forceinline__ bool win_valid(int32_t e) { return (((uint32_t)e) >> 30) != 3u; }

// Prediction stencil (3 x 3, x fastest) of the level-l neighbour at offset
// (ox, oy) from the leaf at (x, y), read from the block: periodic axes wrap
// (the block entries were looked up wrapped), the others take the nearest
// cell of the level, as the prediction operator does at a boundary.
__device__ __forceinline__ bool win_stencil(const Geo& g, int l, int x, int y, int ox, int oy,
                                            const int32_t (*win)[MR_WIN_TPB], int32_t* st) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      int X = ox + i - 1, Y = oy + j - 1;
      if (!g.periodic[0]) {
        const int ax = x + X;
        if (ax < 0) X = -x;
        else if (ax >= g.n[l][0]) X = g.n[l][0] - 1 - x;
      }
      if (!g.periodic[1]) {
        const int ay = y + Y;
        if (ay < 0) Y = -y;
        else if (ay >= g.n[l][1]) Y = g.n[l][1] - 1 - y;
      }
      const int32_t e = win[(Y + 2) * 5 + X + 2][threadIdx.x];
      st[j * 3 + i] = e;
      ok = ok && win_valid(e);
    }
  return ok;
}

template <class Sc, int F>
__device__ __forceinline__ void stream_window_d2(const Geo& g, const MeshDev& B,
                                                 const typename FormT<F>::S* __restrict__ LFin,
                                                 const typename FormT<F>::C* __restrict__ W, int l, int x, int y,
                                                 int i, const typename FormT<F>::C* fs,
                                                 const typename FormT<F>::C* offv, typename FormT<F>::C* out,
                                                 typename FormT<F>::C scale, typename FormT<F>::C* tmp,
                                                 int32_t (*win)[MR_WIN_TPB],
                                                 const typename FormT<F>::C* __restrict__ det) {
  using S = typename FormT<F>::S;
  using C = typename FormT<F>::C;
  const C cs = MR_K(C, g, cross_sign);
  const int tid = threadIdx.x;
  {
    MortonBox<2> bx;
    bx.init(g, l, x, y);
    const int32_t* map = B.map + g.base[l];
    int32_t e[25];
#pragma unroll
    for (int w = 0; w < 25; ++w) {
      const int a = w % 5, b = w / 5;
      if (w == 12)
        e[w] = (int32_t)((MR_CLS_LEAF << 30) | (uint32_t)i);
      else
        e[w] = bx.in(a, b) ? map[bx.code(a, b)] : MR_WIN_OUT;
    }
    bool bad = false;
#pragma unroll
    for (int w = 0; w < 25; ++w) {
      bad = bad || e[w] == MR_MAP_NONE;
      win[w][tid] = e[w];
    }
    if (bad) mr_set_err(B.cnt, MR_DERR_INTERNAL);  // a cell the transport reads is neither in the tree nor a ghost
  }

  // ---- axis strips, boundary values and critical-case corrections
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    ValPtr<S> vp[4];
    bool has[4];
    int32_t ent[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int off = w < 2 ? w - 2 : w - 1;  // -2, -1, +1, +2 along a
      ent[w] = win[a == 0 ? 12 + off : 12 + 5 * off][tid];
      has[w] = win_valid(ent[w]);
      vp[w] = mr_resolve<S>(g, B, LFin, has[w] ? ent[w] : 0);
    }
    stream_axis<Sc, F>(g, B, LFin, W, l, a, x, y, 0, vp, has, ent, fs, offv, out, scale, tmp, win, det);
  }

  // ---- the four single finest cells of each diagonal velocity
  constexpr int P0 = Sc::DIAG0;
  const int Nx = g.n[l][0], Ny = g.n[l][1];
  const int slx = mr_slot(x, Nx, g.periodic[0]), sly = mr_slot(y, Ny, g.periodic[1]);
  const C* wx[2] = {W + MR_WIDX(l, 0, slx, 0), W + MR_WIDX(l, 0, slx, 1)};
  const C* wy[2] = {W + MR_WIDX(l, 1, sly, 0), W + MR_WIDX(l, 1, sly, 1)};
  C acc[4] = {(C)0, (C)0, (C)0, (C)0};
  for (int b = 0; b < 5; ++b) {
    const C wy0 = wy[0][b], wy1 = wy[1][b];
    if (wy0 == (C)0 && wy1 == (C)0) continue;  // zero row: adds nothing
#pragma unroll
    for (int a = 0; a < 5; ++a) {
      const C wx0 = wx[0][a], wx1 = wx[1][a];
      if (wx0 == (C)0 && wx1 == (C)0) continue;
      const int32_t e = win[b * 5 + a][tid];
      const bool self = a == 2 && b == 2;
      if (!self && !win_valid(e)) continue;  // outside: zero weight
      const ValPtr<S> vp = mr_resolve<S>(g, B, LFin, self ? 0 : e);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int p = P0 + t;
        const C wab = (Sc::eta(p, 0) > 0 ? wx0 : wx1) * (Sc::eta(p, 1) > 0 ? wy0 : wy1);
        if (wab == (C)0) continue;
        const C v = self ? fs[p] : ld_off<F>(vp, p, offv);
        acc[t] += wab * v;
      }
    }
  }
  if (l < g.J) {
    for (int nb = 0; nb < 9; ++nb) {
      if (nb == 4) continue;
      const int dx = nb % 3 - 1, dy = nb / 3 - 1;
      const int32_t e = win[(dy + 2) * 5 + dx + 2][tid];
      if (!win_valid(e) || (((uint32_t)e) >> 30) != MR_CLS_INT) continue;
      const uint32_t ridx = (uint32_t)e & 0x3FFFFFFFu;  // its children's details: det (k_edge_details)
      const size_t cap1 = g.cap[1];
      C wcx[2][2], wcy[2][2];  // [sign index][child offset]
#pragma unroll
      for (int si = 0; si < 2; ++si)
#pragma unroll
        for (int o = 0; o < 2; ++o) {
          wcx[si][o] = corner_edge_weight(g, W, l + 1, 0, x, 2 * dx + o, si == 0 ? 1 : -1);
          wcy[si][o] = corner_edge_weight(g, W, l + 1, 1, y, 2 * dy + o, si == 0 ? 1 : -1);
        }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int p = P0 + t;
        const int ix = Sc::eta(p, 0) > 0 ? 0 : 1, iy = Sc::eta(p, 1) > 0 ? 0 : 1;
        C corr = (C)0;
#pragma unroll
        for (int ci = 0; ci < 4; ++ci) {
          const C w = wcx[ix][ci & 1] * wcy[iy][ci >> 1];
          if (w == (C)0) continue;
          corr += w * det[((size_t)ci * Sc::Q + p) * cap1 + ridx];
        }
        acc[t] += corr;
      }
    }
  }
  const C scale2 = scale * scale;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int p = P0 + t;
    const int sx = Sc::eta(p, 0), sy = Sc::eta(p, 1);
    const bool outx = !g.periodic[0] && (sx > 0 ? x == 0 : x == Nx - 1);
    const bool outy = !g.periodic[1] && (sy > 0 ? y == 0 : y == Ny - 1);
    if (outx && outy) acc[t] -= bc_value<C>(g, g.bc[sy > 0 ? 2 : 3], fs, p, Sc::opp(p));
    out[p] += scale2 * acc[t];
  }
}

// ------------------------------------------------------------------ critical-case details (D2Q9)
// The details of the children of every refined cell that a leaf of its own
// level borders (within its 3 x 3 neighbourhood), for every population:
// det[(child * Q + p) * cap_int + i] = child value - its prediction from the
// refined cell's 3 x 3 stencil, in the form's arithmetic, the operations the
// transport would perform.  The transport of a D2Q9 leaf then reads them for
// its refined neighbours (axis strips and diagonal corner cells) instead of
// predicting the children again: each refined cell is done once, not by
// each of up to eight leaves around it, for up to eight populations each.
template <int F>
__global__ void __launch_bounds__(128) k_edge_details(const InstDev* __restrict__ IB, int ngrp, int dst) {
  using S = typename FormT<F>::S;
  using C = typename FormT<F>::C;
  constexpr int Q = Scheme<4>::Q;
  extern __shared__ int pre[];
  __shared__ InstDev si;
  int have = -1;
  mr_inst_prefetch(si, have, IB, ngrp);
  mr_grid_dep();  // after the copy of the descriptor, which no step kernel writes
  const int tiles =
      mr_group_prefix(pre, ngrp, [&](int b) { return (IB[b].mesh[dst].cnt->total[MR_CLS_INT] + 127) / 128; });
  for (int tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
    const int b = mr_group_find(pre, ngrp, tt);
    mr_inst_use(si, have, IB, b);
    const Geo& g = si.g;
    const MeshDev& B = si.mesh[dst];
    const int i = (tt - pre[b]) * 128 + threadIdx.x;
    if (i >= B.cnt->total[MR_CLS_INT]) continue;
    const int l = B.lvl[MR_CLS_INT][i];
    const uint32_t code = B.code[MR_CLS_INT][i];
    int x, y;
    mr_decode(g, l, code, x, y);
    // does a leaf of level l border it?
    MortonBox<1> bx;
    bx.init(g, l, x, y);
    const int32_t* map = B.map + g.base[l];
    bool need = false;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      if (k == 4 || !bx.in(k % 3, k / 3)) continue;
      const int32_t e = map[bx.code(k % 3, k / 3)];
      need = need || (e != MR_MAP_NONE && (((uint32_t)e) >> 30) == MR_CLS_LEAF);
    }
    if (!need) continue;
    int32_t st[9], ce[4];
    bool ok = mr_stencil_entries<2>(g, B, l, x, y, st);
#pragma unroll
    for (int ci = 0; ci < 4; ++ci) {
      ce[ci] = B.map[g.base[l + 1] + ((code << 2) | (uint32_t)ci)];
      ok = ok && ce[ci] != MR_MAP_NONE;
    }
    if (!ok) {
      mr_set_err(B.cnt, MR_DERR_INTERNAL);
      continue;
    }
    const S* LFin = (const S*)si.fscratch;
    C* det = (C*)si.det;
    const C cs = MR_K(C, g, cross_sign);
    const size_t cap1 = g.cap[1];
#pragma unroll 1
    for (int p = 0; p < Q; ++p) {
      C v[9];
#pragma unroll
      for (int kk = 0; kk < 9; ++kk) v[kk] = ld_c<C>(mr_resolve<S>(g, B, LFin, st[kk]), p);
#pragma unroll
      for (int ci = 0; ci < 4; ++ci)
        det[((size_t)ci * Q + p) * cap1 + i] =
            ld_c<C>(mr_resolve<S>(g, B, LFin, ce[ci]), p) - predict_c<2, C>(v, ci, cs);
    }
  }
}

// ------------------------------------------------------------------ transport + collision
template <int SC, int F>
__global__ void __launch_bounds__(MR_WIN_TPB) k_stream_collide(const InstDev* __restrict__ IB, int ngrp, int dst,
                                                        int do_stream, int do_collide, int count) {
  using Sc = Scheme<SC>;
  using S = typename FormT<F>::S;
  using C = typename FormT<F>::C;
  constexpr bool OFFS = FormT<F>::offs;
  constexpr int D = Sc::D, Q = Sc::Q;
  extern __shared__ int pre[];
  __shared__ InstDev si;
  // per-thread buffers: the leaf's populations and the rolled loops' terms
  constexpr int STR = ThreadStride<Q>::value;
  __shared__ C fsh[MR_WIN_TPB * STR], tsh[MR_WIN_TPB * STR];
  C* fs = fsh + threadIdx.x * STR;
  C* tmp = tsh + threadIdx.x * STR;
  int have = -1;
  mr_inst_prefetch(si, have, IB, ngrp);
  mr_grid_dep();  // after the copy of the descriptor, which no step kernel writes
  const int tiles =
      mr_group_prefix(pre, ngrp, [&](int b) {
        return (IB[b].mesh[dst].cnt->total[MR_CLS_LEAF] + MR_WIN_TPB - 1) / MR_WIN_TPB;
      });
  for (int tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
    const int b = mr_group_find(pre, ngrp, tt);
    mr_inst_use(si, have, IB, b);
    const Geo& g = si.g;
    const MeshDev& B = si.mesh[dst];
    const S* __restrict__ LFin = (const S*)si.fscratch;
    S* __restrict__ LFout = (S*)si.fstate;
    const C* __restrict__ W = mr_wtab<C>(si);
    const int i = (tt - pre[b]) * MR_WIN_TPB + threadIdx.x;
    if (count && tt == pre[b] && threadIdx.x == 0) {
      // the step's counters (leaf updates, steps), once per instance
      B.cnt->leaf_updates += B.cnt->total[MR_CLS_LEAF];
      B.cnt->steps += 1;
    }
    if (i >= B.cnt->total[MR_CLS_LEAF]) continue;
    const int l = B.lvl[MR_CLS_LEAF][i];
    const uint32_t code = B.code[MR_CLS_LEAF][i];
    // the leaf's own populations stay in shared memory (fs) beside the
    // register accumulators, and the storage offsets are read where used
    const C* offv = mr_offv<C>(g);
    C out[Q];
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      ValPtr<S> me{LFin + i, g.cap[0]};
      out[p] = ld_off<F>(me, p, offv);
      fs[p] = out[p];
    }
    if (do_stream) {
      int xc[3] = {0, 0, 0};
      mr_decode_d<D>(g, l, code, xc);
      const int x = xc[0], y = xc[1], z = xc[2];
      const C scale = (C)__longlong_as_double((long long)(1023 + l - g.J) << 52);  // 2^{l-J}, exact
      if constexpr (Sc::DIAG) {
        __shared__ int32_t win[25][MR_WIN_TPB];
        stream_window_d2<Sc, F>(g, B, LFin, W, l, x, y, i, fs, offv, out, scale, tmp, win, (const C*)si.det);
      } else {
#pragma unroll
        for (int a = 0; a < D; ++a) {
          ValPtr<S> vp[4];
          bool has[4];
          int32_t ent[4];
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int off = w < 2 ? w - 2 : w - 1;  // -2, -1, +1, +2 along a
            int nb[3] = {x, y, z};
            nb[a] += off;
            has[w] = mr_nbr_mesh_d<D>(g, l, nb);
            ent[w] = has[w] ? B.map[g.base[l] + mr_encode_d<D>(g, l, nb)] : MR_MAP_NONE;
            if (has[w] && ent[w] == MR_MAP_NONE) {
              mr_set_err(B.cnt, MR_DERR_INTERNAL);
              has[w] = false;
            }
            vp[w] = mr_resolve<S>(g, B, LFin, has[w] ? ent[w] : 0);
          }
          stream_axis<Sc, F>(g, B, LFin, W, l, a, x, y, z, vp, has, ent, fs, offv, out, scale, tmp, nullptr);
        }
      }
    }
    if (do_collide) {
      Sc::template collide<C>(g, out);
      if constexpr (Sc::DIAG) {
        if (g.obstacle) {
          const double phi = obstacle_fraction(g, l, code);
          if (phi > 0.0) {
#pragma unroll
            for (int p = 0; p < Q; ++p) out[p] = (C)phi * MR_K(C, g, feq0[p]) + ((C)1 - (C)phi) * out[p];
          }
        }
      }
    }
    bool finite = true;
#pragma unroll
    for (int p = 0; p < Q; ++p) {
      finite = finite && is_finite_bits(out[p]);
      if constexpr (OFFS)
        LFout[(size_t)p * g.cap[0] + i] = mr_from_f<S>((float)(out[p] - offv[p]));
      else
        LFout[(size_t)p * g.cap[0] + i] = (S)out[p];
    }
    if (!finite) mr_set_err(B.cnt, MR_DERR_NONFINITE);
  }
}

// ------------------------------------------------------------------ input / output
template <int SC, int F>
__global__ void __launch_bounds__(256) k_init_eq(Geo g, MeshDev B, const double* __restrict__ cons, void* LF_) {
  using Sc = Scheme<SC>;
  using S = typename FormT<F>::S;
  S* LF = (S*)LF_;
  const int n = B.cnt->total[MR_CLS_LEAF];
  const long long NJ = (long long)g.n[g.J][0] * g.n[g.J][1] * g.n[g.J][2];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int c[3] = {0, 0, 0};
    mr_decode_d<Sc::D>(g, g.J, B.code[MR_CLS_LEAF][i], c);
    const long long r = ((long long)c[2] * g.n[g.J][1] + c[1]) * g.n[g.J][0] + c[0];
    double u[4], f[Sc::Q];
    for (int k = 0; k < g.ncons; ++k) u[k] = cons[k * NJ + r];
    Sc::equilibrium(g, u, f);
#pragma unroll
    for (int p = 0; p < Sc::Q; ++p)
      LF[(size_t)p * g.cap[0] + i] = mr_from_d<S>(FormT<F>::offs ? f[p] - g.off[p] : f[p]);
  }
}

template <int F>
__global__ void __launch_bounds__(256) k_gather_input(Geo g, MeshDev B, const int32_t* __restrict__ inidx,
                                                      long long nin, const double* __restrict__ fin, void* LF_) {
  using S = typename FormT<F>::S;
  S* LF = (S*)LF_;
  const int n = B.cnt->total[MR_CLS_LEAF];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int l = B.lvl[MR_CLS_LEAF][i];
    const int32_t j = inidx[g.base[l] + B.code[MR_CLS_LEAF][i]];
    if (j < 0 || j >= nin) {
      mr_set_err(B.cnt, MR_DERR_INPUT);
      continue;
    }
    for (int p = 0; p < g.Q; ++p) {
      const double v = fin[(size_t)p * nin + j];
      LF[(size_t)p * g.cap[0] + i] = mr_from_d<S>(FormT<F>::offs ? v - g.off[p] : v);
    }
  }
}

template <int F>
__global__ void __launch_bounds__(256) k_leaves_out(Geo g, MeshDev B, const void* __restrict__ LF_, long long n,
                                                    unsigned long long* keys, signed char* levels, double* f) {
  using S = typename FormT<F>::S;
  const S* LF = (const S*)LF_;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (keys) keys[i] = B.code[MR_CLS_LEAF][i];
    if (levels) levels[i] = (signed char)B.lvl[MR_CLS_LEAF][i];
    if (f)
      for (int p = 0; p < g.Q; ++p) {
        const double v = mr_cvt_d(LF[(size_t)p * g.cap[0] + i]);
        f[(size_t)p * n + i] = FormT<F>::offs ? v + g.off[p] : v;
      }
  }
}

// Conserved moments on the uniform level `level`, row-major: values of the
// complete tree where present, the prediction of the level above otherwise.
template <int D, int F>
__global__ void __launch_bounds__(256) k_project_dense(Geo g, MeshDev B, const void* __restrict__ LF, int level,
                                                       const double* __restrict__ prev, double* cur) {
  using S = typename FormT<F>::S;
  constexpr int NS = Pow3<D>::value;
  const int n0 = g.n[level][0], n1 = g.n[level][1];
  const long long N = (long long)n0 * n1 * g.n[level][2];
  const int p0 = level > g.Jmin ? g.n[level - 1][0] : 1, p1 = level > g.Jmin ? g.n[level - 1][1] : 1;
  const long long PN = level > g.Jmin ? (long long)p0 * p1 * g.n[level - 1][2] : 1;
  const double cs = (double)g.cross_sign;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
       r += (long long)gridDim.x * blockDim.x) {
    const int c[3] = {(int)(r % n0), (int)((r / n0) % n1), (int)(r / ((long long)n0 * n1))};
    const int32_t e = B.map[g.base[level] + mr_encode_d<D>(g, level, c)];
    if (e != MR_MAP_NONE && (((uint32_t)e) >> 30) <= MR_CLS_INT) {
      const ValPtr<S> v = mr_resolve<S>(g, B, LF, e);
      for (int k = 0; k < g.ncons; ++k) {
        double acc = 0.0;
        for (int p = 0; p < g.Q; ++p)
          acc += g.consw[k][p] * (mr_ld(v, p) + (FormT<F>::offs ? g.off[p] : 0.0));
        cur[k * N + r] = acc;
      }
    } else if (level > g.Jmin) {
      int ci = 0;
      for (int a = 0; a < D; ++a) ci |= (c[a] & 1) << a;
      for (int k = 0; k < g.ncons; ++k) {
        double v[NS];
        for (int q = 0; q < NS; ++q) {
          int s[3] = {(c[0] >> 1) + q % 3 - 1, D >= 2 ? (c[1] >> 1) + (q / 3) % 3 - 1 : 0,
                      D == 3 ? (c[2] >> 1) + q / 9 - 1 : 0};
          mr_nbr_stencil_d<D>(g, level - 1, s);
          v[q] = prev[k * PN + ((long long)s[2] * p1 + s[1]) * p0 + s[0]];
        }
        if constexpr (D == 3)
          cur[k * N + r] = predict_c<3, double>(v, ci, cs);
        else
          cur[k * N + r] = mr_predict_fast<D>(v, ci, cs);
      }
    } else {
      mr_set_err(B.cnt, MR_DERR_INTERNAL);
    }
  }
}

template <int Q, int F>
void launch_remesh_t(const Group& G, int cur, cudaStream_t st) {
  mr_launch_pdl(k_remesh_copy<Q, F>, mr_tile_grid(G, G.capL + G.capI, 32, G.bps[MR_PH_REMESH]), dim3(32, PopRows<Q>::value),
                mr_pre_bytes(G), st, G.dev, G.n, cur);
}
template <int D, int Q, int F>
void launch_predict_t(const Group& G, int dst, int kl, cudaStream_t st) {
  // ghosts and leaves of one level: at most twice its cells
  mr_launch_pdl(k_predict_level<D, Q, F>, mr_tile_grid(G, 2 * G.pred_cells[kl], 32, G.bps[MR_PH_PREDICT]), dim3(32, PopRows<Q>::value),
                mr_pre_bytes(G), st, G.dev, G.n, dst, kl);
}
template <int F>
void launch_edge_t(const Group& G, int dst, cudaStream_t st) {
  mr_launch_pdl(k_edge_details<F>, mr_tile_grid(G, G.capI, 128, G.bps[MR_PH_STREAM]), 128, mr_pre_bytes(G), st, G.dev,
                G.n, dst);
}
template <int SC, int F>
void launch_stream_t(const Group& G, int dst, int ds, int dc, int count, cudaStream_t st) {
  mr_launch_pdl(k_stream_collide<SC, F>, mr_tile_grid(G, G.capL, MR_WIN_TPB, G.bps[MR_PH_STREAM]), MR_WIN_TPB, mr_pre_bytes(G), st, G.dev,
                G.n, dst, ds, dc, count);
}
template <int SC, int F>
void launch_init_t(const Geo& g, const MeshDev& B, const double* cons, void* LF, cudaStream_t st, int grid) {
  k_init_eq<SC, F><<<grid, 256, 0, st>>>(g, B, cons, LF);
}

}  // namespace

#define MR_FORMS(FN, ...)                                          \
  switch (G.form) {                                                \
    case MR_FORM_F64: FN<MR_FORM_F64>(__VA_ARGS__); break;         \
    case MR_FORM_F32: FN<MR_FORM_F32>(__VA_ARGS__); break;         \
    case MR_FORM_F32_F16: FN<MR_FORM_F32_F16>(__VA_ARGS__); break; \
    case MR_FORM_F32_BF16: FN<MR_FORM_F32_BF16>(__VA_ARGS__); break; \
  }
#define MR_FORMS2(FN, A1, ...)                                         \
  switch (G.form) {                                                    \
    case MR_FORM_F64: FN<A1, MR_FORM_F64>(__VA_ARGS__); break;         \
    case MR_FORM_F32: FN<A1, MR_FORM_F32>(__VA_ARGS__); break;         \
    case MR_FORM_F32_F16: FN<A1, MR_FORM_F32_F16>(__VA_ARGS__); break; \
    case MR_FORM_F32_BF16: FN<A1, MR_FORM_F32_BF16>(__VA_ARGS__); break; \
  }
#define MR_FORMS3(FN, A1, A2, ...)                                         \
  switch (G.form) {                                                        \
    case MR_FORM_F64: FN<A1, A2, MR_FORM_F64>(__VA_ARGS__); break;         \
    case MR_FORM_F32: FN<A1, A2, MR_FORM_F32>(__VA_ARGS__); break;         \
    case MR_FORM_F32_F16: FN<A1, A2, MR_FORM_F32_F16>(__VA_ARGS__); break; \
    case MR_FORM_F32_BF16: FN<A1, A2, MR_FORM_F32_BF16>(__VA_ARGS__); break; \
  }

size_t mr_form_bytes(int form) {
  switch (form) {
    case MR_FORM_F64: return 8;
    case MR_FORM_F32: return 4;
    default: return 2;
  }
}

void mr_launch_remesh_copy(const Group& G, int cur, cudaStream_t st) {
  switch (G.Q) {
    case 2: MR_FORMS2(launch_remesh_t, 2, G, cur, st); break;
    case 3: MR_FORMS2(launch_remesh_t, 3, G, cur, st); break;
    case 9: MR_FORMS2(launch_remesh_t, 9, G, cur, st); break;
    case 16: MR_FORMS2(launch_remesh_t, 16, G, cur, st); break;
    case 6: MR_FORMS2(launch_remesh_t, 6, G, cur, st); break;
  }
}

void mr_launch_predict_level(const Group& G, int dst, int kl, cudaStream_t st) {
  if (G.s > 1) return mr_launch_predict_level_w(G, dst, kl, st);
  switch (G.d * 100 + G.Q) {
    case 102: MR_FORMS3(launch_predict_t, 1, 2, G, dst, kl, st); break;
    case 103: MR_FORMS3(launch_predict_t, 1, 3, G, dst, kl, st); break;
    case 209: MR_FORMS3(launch_predict_t, 2, 9, G, dst, kl, st); break;
    case 216: MR_FORMS3(launch_predict_t, 2, 16, G, dst, kl, st); break;
    case 306: MR_FORMS3(launch_predict_t, 3, 6, G, dst, kl, st); break;
  }
}

void mr_launch_stream_collide(const Group& G, int dst, int do_stream, int do_collide, cudaStream_t st,
                              int count) {
  if (G.s > 1) return mr_launch_stream_collide_w(G, dst, do_stream, do_collide, st, count);
  switch (G.scheme) {
    case 0: MR_FORMS2(launch_stream_t, 0, G, dst, do_stream, do_collide, count, st); break;
    case 1: MR_FORMS2(launch_stream_t, 1, G, dst, do_stream, do_collide, count, st); break;
    case 2: MR_FORMS2(launch_stream_t, 2, G, dst, do_stream, do_collide, count, st); break;
    case 3: MR_FORMS2(launch_stream_t, 3, G, dst, do_stream, do_collide, count, st); break;
    case 4: MR_FORMS2(launch_stream_t, 4, G, dst, do_stream, do_collide, count, st); break;
    case 5: MR_FORMS2(launch_stream_t, 5, G, dst, do_stream, do_collide, count, st); break;
  }
}

void mr_launch_edge_details(const Group& G, int dst, cudaStream_t st) { MR_FORMS(launch_edge_t, G, dst, st); }

void mr_launch_init_eq(const Geo& g, const MeshDev& B, const double* cons, void* LF, cudaStream_t st, int grid) {
  const Geo& G = g;
  switch (g.scheme) {
    case 0: MR_FORMS2(launch_init_t, 0, g, B, cons, LF, st, grid); break;
    case 1: MR_FORMS2(launch_init_t, 1, g, B, cons, LF, st, grid); break;
    case 2: MR_FORMS2(launch_init_t, 2, g, B, cons, LF, st, grid); break;
    case 3: MR_FORMS2(launch_init_t, 3, g, B, cons, LF, st, grid); break;
    case 4: MR_FORMS2(launch_init_t, 4, g, B, cons, LF, st, grid); break;
    case 5: MR_FORMS2(launch_init_t, 5, g, B, cons, LF, st, grid); break;
  }
}

template <int F>
static void launch_gather_t(const Geo& g, const MeshDev& B, const int32_t* inidx, long long n, const double* fin,
                            void* LF, cudaStream_t st, int grid) {
  k_gather_input<F><<<grid, 256, 0, st>>>(g, B, inidx, n, fin, LF);
}
void mr_launch_gather_input(const Geo& g, const MeshDev& B, const int32_t* inidx, long long n, const double* fin,
                            void* LF, cudaStream_t st, int grid) {
  const Geo& G = g;
  MR_FORMS(launch_gather_t, g, B, inidx, n, fin, LF, st, grid);
}

template <int F>
static void launch_out_t(const Geo& g, const MeshDev& B, const void* LF, long long n, unsigned long long* keys,
                         signed char* levels, double* f, cudaStream_t st, int grid) {
  k_leaves_out<F><<<grid, 256, 0, st>>>(g, B, LF, n, keys, levels, f);
}
void mr_launch_leaves_out(const Geo& g, const MeshDev& B, const void* LF, long long n, unsigned long long* keys,
                          signed char* levels, double* f, cudaStream_t st, int grid) {
  const Geo& G = g;
  MR_FORMS(launch_out_t, g, B, LF, n, keys, levels, f, st, grid);
}

template <int D, int F>
static void launch_dense_t(const Geo& g, const MeshDev& B, const void* LF, int level, const double* prev,
                           double* cur, cudaStream_t st, int grid) {
  k_project_dense<D, F><<<grid, 256, 0, st>>>(g, B, LF, level, prev, cur);
}
void mr_launch_project_dense(const Geo& g, const MeshDev& B, const void* LF, int level, const double* prev,
                             double* cur, cudaStream_t st, int grid) {
  if (g.s_pred > 1) return mr_launch_project_dense_w(g, B, LF, level, prev, cur, st, grid);
  const Geo& G = g;
  if (g.d == 1) {
    MR_FORMS2(launch_dense_t, 1, g, B, LF, level, prev, cur, st, grid);
  } else if (g.d == 2) {
    MR_FORMS2(launch_dense_t, 2, g, B, LF, level, prev, cur, st, grid);
  } else {
    MR_FORMS2(launch_dense_t, 3, g, B, LF, level, prev, cur, st, grid);
  }
}


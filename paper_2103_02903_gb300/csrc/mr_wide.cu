// The adaptive step with the prediction operator of half-width s = 2, 3
// (Table 1; the tensor-product operators of Sec. 4.1 for d = 2, 3).
//
// What changes with s, phase by phase:
// - details (Def. Details): each internal cell predicts its 2^d children
//   from its (2s+1)^d stencil; the evaluation order is the one of the
//   operator's written form (axis sums, then the pair and triple diagonal
//   sums, each started from its (1, 1, 1) term), in FP64 without
//   contraction, so the group norms carry the same bits as a plain
//   evaluation of those formulas;
// - grading (Def. Grading): the parent of every tree cell has its
//   (2s+1)^d neighbourhood in the tree;
// - ghosts: the transport window reaches W = 2s cells on either side of a
//   leaf along each axis, and every ghost's parent has its (2s+1)^d stencil
//   available (tree cells or ghosts, cascading towards J_min);
// - transport (Eq. AdaptiveAdvectionPhase with Eq. PredictionWithMatrixNew):
//   the row-collapsed sums are the flattened weights of half-width W
//   applied to the leaf's row, and every refined cell of the window adds the
//   details of its children through the level-(j+1) edge weights (the
//   critical case of Sec. 6.1).  Grading with radius s keeps level j+2
//   cells out of reach of the leaf's edge reconstruction: a level-(j+2)
//   cell below a level-(j+1) cell c needs c's +-s neighbourhood in the tree,
//   which excludes the leaf's own children, so such cells lie 2s or more
//   level-(j+2) cells away from the leaf's faces, beyond the W = 2s window.
// Lattices with diagonal velocities (D2Q9) add the four corner cells of each
// diagonal velocity over the (2W+1)^2 block around the leaf.
//
// The tuned s = 1 kernels are untouched; these are plain one-thread-per-cell
// kernels that look cells up through the dense index map.
#include "mr_wide.cuh"

namespace {

// Map entries of the (2s+1)^D stencil around cell c of level l (constant
// extension outside a non-periodic domain, wrap on a periodic axis).
template <int D, int S>
__device__ __forceinline__ bool wide_stencil(const Geo& g, const MeshDev& M, int l, const int* c, int32_t* ent) {
  using B = WBox<D, S>;
  bool ok = true;
  for (int k = 0; k < B::N; ++k) {
    int s[3] = {c[0] + k % B::W1 - S, D >= 2 ? c[1] + (k / B::W1) % B::W1 - S : 0,
                D == 3 ? c[2] + k / (B::W1 * B::W1) - S : 0};
    mr_nbr_stencil_d<D>(g, l, s);
    ent[k] = M.map[g.base[l] + mr_encode_d<D>(g, l, s)];
    ok = ok && ent[k] != MR_MAP_NONE;
  }
  return ok;
}

// Entry k (x fastest) of the (2s+1)^D stencil around cell c of level l.
template <int D, int S>
__device__ __forceinline__ int32_t wide_stencil_entry(const Geo& g, const MeshDev& M, int l, const int* c, int k) {
  using B = WBox<D, S>;
  int s[3] = {c[0] + k % B::W1 - S, D >= 2 ? c[1] + (k / B::W1) % B::W1 - S : 0,
              D == 3 ? c[2] + k / (B::W1 * B::W1) - S : 0};
  mr_nbr_stencil_d<D>(g, l, s);
  return M.map[g.base[l] + mr_encode_d<D>(g, l, s)];
}

// Thread layout of the wide details and prediction kernels: a tile of TC
// cells (threadIdx.x) by 8 population rows (threadIdx.y); the rows share one
// lookup of each cell's stencil (and children) through shared memory.
template <int D, int S>
struct WTile {
  static constexpr int TC = (D == 3 && S == 3) ? 16 : 32;  // 343-cell stencils: half the cells per tile
};

// ------------------------------------------------------------------ details
// Group norm of the details of every internal cell's children (Def. Details,
// max over the 2^d children and all populations), FP64 on stored values.
template <int D, int S, int F>
__global__ void __launch_bounds__(256) k_details_w(const InstDev* __restrict__ IB, int n, int cur) {
  using St = typename FormT<F>::S;
  using B = WBox<D, S>;
  constexpr int TC = WTile<D, S>::TC, NE = B::N + (1 << D);
  extern __shared__ int pre[];
  __shared__ InstDev si;
  __shared__ int32_t sent[NE][TC];
  __shared__ double red[8][TC];
  int have = -1;
  mr_inst_prefetch(si, have, IB, n);
  mr_grid_dep();
  const int tiles =
      mr_group_prefix(pre, n, [&](int b) { return (IB[b].mesh[cur].cnt->total[MR_CLS_INT] + TC - 1) / TC; });
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {  // uniform over the block
    const int b = mr_group_find(pre, n, t);
    mr_inst_use(si, have, IB, b);
    const Geo& g = si.g;
    const MeshDev& A = si.mesh[cur];
    const int nI = A.cnt->total[MR_CLS_INT];
    const int i = (t - pre[b]) * TC + tx;
    if (i < nI) {
      const int L = A.lvl[MR_CLS_INT][i];
      const uint32_t code = A.code[MR_CLS_INT][i];
      int c[3] = {0, 0, 0};
      mr_decode_d<D>(g, L, code, c);
      for (int e = ty; e < NE; e += 8)
        sent[e][tx] = e < B::N ? wide_stencil_entry<D, S>(g, A, L, c, e)
                               : A.map[g.base[L + 1] + ((code << D) | (uint32_t)(e - B::N))];
    }
    __syncthreads();
    double gmax = 0.0;
    bool ok = i < nI;
    if (ok) {
      for (int e = 0; e < NE; ++e) {
        const int32_t en = sent[e][tx];
        ok = ok && en != MR_MAP_NONE && (((uint32_t)en) >> 30) <= MR_CLS_INT;
      }
      if (!ok) {
        if (ty == 0) mr_set_err(A.cnt, MR_DERR_INTERNAL);
      } else {
        for (int p = ty; p < g.Q; p += 8) {
          double v[B::N];
          for (int k = 0; k < B::N; ++k) v[k] = mr_ld(mr_resolve<St>(g, A, si.fstate, sent[k][tx]), p);
#pragma unroll 1
          for (int ci = 0; ci < (1 << D); ++ci) {
            const double pr = wide_predict<D, S, double, true>(v, ci, g.cross_sign);
            const double d = fabs(__dsub_rn(mr_ld(mr_resolve<St>(g, A, si.fstate, sent[B::N + ci][tx]), p), pr));
            gmax = d > gmax ? d : gmax;
          }
        }
      }
    }
    red[ty][tx] = gmax;
    __syncthreads();
    if (ty == 0 && ok) {
      double m = red[0][tx];
      for (int r = 1; r < 8; ++r) m = red[r][tx] > m ? red[r][tx] : m;
      A.G[i] = m;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ grading
// Every cell refined after H_eps (or by the grading itself) needs the
// (2s+1)^D cells around it in the tree: their parents are marked refined,
// depth first towards J_min by the thread that marks them first.
template <int D, int S>
__global__ void __launch_bounds__(256) k_grade_w(const InstDev* __restrict__ IB, int n) {
  using B = WBox<D, S>;
  extern __shared__ int pre[];
  __shared__ InstDev si;
  int have = -1;
  mr_inst_prefetch(si, have, IB, n);
  mr_grid_dep();
  const int tiles = mr_group_prefix(pre, n, [&](int b) {
    const Geo& gb = IB[b].g;
    return gb.J > gb.Jmin + 1 ? (int)((gb.base[gb.J] - gb.base[gb.Jmin + 1] + 255) / 256) : 0;
  });
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int b = mr_group_find(pre, n, t);
    mr_inst_use(si, have, IB, b);
    const Geo& g = si.g;
    uint8_t* flags = si.flags;
    const uint32_t t0 = g.base[g.Jmin + 1] + (uint32_t)(t - pre[b]) * 256u, gi = t0 + threadIdx.x;
    if (!si.acth[t0 / MR_DENSE_ALIGN]) continue;  // no H flag in this tile's chunk
    if (gi >= g.base[g.J]) continue;
    if (!(flags[gi] & MR_F_H)) continue;
    const int l0 = mr_level_of(g, gi);
    const uint32_t c0 = gi - g.base[l0];
    if (c0 >= g.ncode[l0]) continue;
    int sl[MR_MAXL], sc[MR_MAXL][3], sk[MR_MAXL];
    int sp = 1;
    sl[0] = l0;
    sk[0] = 0;
    sc[0][0] = sc[0][1] = sc[0][2] = 0;
    mr_decode_d<D>(g, l0, c0, sc[0]);
    while (sp > 0) {
      const int f = sp - 1;
      if (sk[f] == B::N) {
        --sp;
        continue;
      }
      const int k = sk[f]++;
      const int L = sl[f];
      int nb[3] = {sc[f][0] + k % B::W1 - S, D >= 2 ? sc[f][1] + (k / B::W1) % B::W1 - S : 0,
                   D == 3 ? sc[f][2] + k / (B::W1 * B::W1) - S : 0};
      if (!mr_nbr_mesh_d<D>(g, L, nb)) continue;
      for (int a = 0; a < D; ++a) nb[a] >>= 1;
      const int tl = L - 1;
      const uint32_t pc = mr_encode_d<D>(g, tl, nb), pi = g.base[tl] + pc;
      if (flags[pi] & (MR_F_H | MR_F_G)) continue;  // plain load first
      const uint32_t old = mr_atomic_or_byte(flags, pi, MR_F_G);
      if (!(old & (MR_F_H | MR_F_G))) {  // the cell and its children's chunk hold cells of the new tree
        mr_touch(si.act, pi);
        mr_touch(si.act, g.base[tl + 1] + (pc << D));
      }
      if (!(old & (MR_F_H | MR_F_G)) && tl > g.Jmin && sp < MR_MAXL) {
        sl[sp] = tl;
        sk[sp] = 0;
        for (int a = 0; a < 3; ++a) sc[sp][a] = a < D ? nb[a] : 0;
        ++sp;
      }
    }
  }
}

// ------------------------------------------------------------------ ghosts
// Cells the transport of a leaf reads that are not in the tree: the window
// of W = 2s cells on either side along each axis, and for a lattice with
// diagonal velocities the whole (2W+1)^2 block around the leaf.  Each one
// not yet marked becomes a ghost, and its parent's (2s+1)^D stencil is
// marked the same way (cells outside the tree become ghosts), towards J_min.
template <int D, int S>
__global__ void __launch_bounds__(256) k_mark_ghosts_w(const InstDev* __restrict__ IB,
                                                       const int* __restrict__ chunk_pre, int n, int nchunks) {
  using B = WBox<D, S>;
  constexpr int W = 2 * S;
  __shared__ InstDev si;
  __shared__ int32_t qc[D][MR_DENSE_ALIGN];  // the chunk's leaves: their coordinates, decoded once
  __shared__ int qn;
  int have = -1;
  mr_grid_dep();
  // a block per touched chunk at a time (a chunk nothing touched holds no leaf)
  for (int t = blockIdx.x; t < nchunks; t += gridDim.x) {
    int chunk;
    const int ib = mr_group_chunk_of(chunk_pre, n, t, chunk);
    if (!__syncthreads_or(threadIdx.x == 0 && IB[ib].act[chunk])) continue;  // one read for the block
    mr_inst_use(si, have, IB, ib);
    const Geo& g = si.g;
    uint8_t* cls = si.cls;
    const uint32_t c0 = (uint32_t)chunk * MR_DENSE_ALIGN;
    const int l = mr_level_of(g, c0);
    const uint32_t cb = c0 - g.base[l];
    if (threadIdx.x == 0) qn = 0;
    __syncthreads();
    // the leaves are a few per cent of the cells: gather them, then spread the
    // (leaf, window cell) pairs over the whole block (the marks are a union of
    // atomic ORs, so the order does not matter)
    {
      const int lane = threadIdx.x & 31;
      for (int k = 0; k < (int)(MR_DENSE_ALIGN / 256u); ++k) {
        const uint32_t off = (uint32_t)k * 256u + threadIdx.x;
        const bool leaf = cb + off < g.ncode[l] && (cls[c0 + off] & 3u) == MR_C_LEAF;
        const uint32_t bal = __ballot_sync(0xffffffffu, leaf);
        int at = 0;
        if (lane == 0 && bal) at = atomicAdd(&qn, __popc(bal));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (leaf) {
          const int q = at + __popc(bal & ((1u << lane) - 1u));
          int c[3] = {0, 0, 0};
          mr_decode_d<D>(g, l, cb + off, c);
          for (int a = 0; a < D; ++a) qc[a][q] = c[a];
        }
      }
    }
    __syncthreads();
    const bool block = D == 2 && g.diag;
    const int nw = block ? (2 * W + 1) * (2 * W + 1) : D * 2 * W;
    const int items = qn * nw;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
      const int w = it % nw;
      if (block && w == (2 * W + 1) * W + W) continue;  // the leaf itself
      const int q = it / nw;
      int nb[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) nb[a] = qc[a][q];
      if (block) {
        nb[0] += w % (2 * W + 1) - W;
        nb[1] += w / (2 * W + 1) - W;
      } else {
        const int axis = w / (2 * W), o = w % (2 * W);
        nb[axis] += o < W ? o - W : o - W + 1;  // -W..-1, 1..W
      }
      if (!mr_nbr_mesh_d<D>(g, l, nb)) continue;
      const uint32_t gw = g.base[l] + mr_encode_d<D>(g, l, nb);
      if (cls[gw] & (3u | MR_C_GHOST)) continue;  // in the tree or marked
      const uint32_t old = mr_atomic_or_byte(cls, gw, MR_C_GHOST);
      if (old & (3u | MR_C_GHOST)) continue;
      mr_touch(si.act, gw);
      if (l - 1 < g.Jmin) continue;
      // cascade over the stencils of the ghosts' parents, each stencil
      // walked by the thread that claims it first
      int sl[MR_MAXL], sc[MR_MAXL][3], sk[MR_MAXL];
      int sp = 1;
      sl[0] = l - 1;
      sk[0] = 0;
      for (int a = 0; a < 3; ++a) sc[0][a] = a < D ? nb[a] >> 1 : 0;
      if (!mr_claim_stencil(cls, si.act, g.base[l - 1] + mr_encode_d<D>(g, l - 1, sc[0]))) continue;
      while (sp > 0) {
        const int f = sp - 1;
        if (sk[f] == B::N) {
          --sp;
          continue;
        }
        const int kk = sk[f]++;
        const int L = sl[f];
        int ac[3] = {sc[f][0] + kk % B::W1 - S, D >= 2 ? sc[f][1] + (kk / B::W1) % B::W1 - S : 0,
                     D == 3 ? sc[f][2] + kk / (B::W1 * B::W1) - S : 0};
        if (!mr_nbr_mesh_d<D>(g, L, ac)) continue;  // outside: the stencil clamps to a cell of the box
        const uint32_t ga = g.base[L] + mr_encode_d<D>(g, L, ac);
        if (cls[ga] & (3u | MR_C_GHOST)) continue;
        const uint32_t o2 = mr_atomic_or_byte(cls, ga, MR_C_GHOST);
        if (o2 & (3u | MR_C_GHOST)) continue;
        mr_touch(si.act, ga);
        if (L - 1 < g.Jmin || sp >= MR_MAXL) continue;
        for (int a = 0; a < 3; ++a) sc[sp][a] = a < D ? ac[a] >> 1 : 0;
        if (!mr_claim_stencil(cls, si.act, g.base[L - 1] + mr_encode_d<D>(g, L - 1, sc[sp]))) continue;
        sl[sp] = L - 1;
        sk[sp] = 0;
        ++sp;
      }
    }
  }  // the barrier at the top of the next chunk ends this chunk's use of the queue
}

// ------------------------------------------------------------------ prediction of ghosts and new leaves
// Ghosts and newly created leaves of level J_min + kl: the prediction of
// half-width s applied to the level-1 values of the new mesh.
template <int D, int S, int F>
__global__ void __launch_bounds__(256) k_predict_level_w(const InstDev* __restrict__ IB, int ngrp, int dst, int kl) {
  using St = typename FormT<F>::S;
  using C = typename FormT<F>::C;
  using B = WBox<D, S>;
  constexpr int TC = WTile<D, S>::TC;
  extern __shared__ int pre[];
  __shared__ InstDev si;
  __shared__ int32_t sent[B::N][TC];
  int have = -1;
  mr_inst_prefetch(si, have, IB, ngrp);
  mr_grid_dep();
  const int tiles = mr_group_prefix(pre, ngrp, [&](int b) {
    const Geo& gb = IB[b].g;
    const int l = gb.Jmin + kl;
    if (l > gb.J) return 0;
    const MeshCounts* c = IB[b].mesh[dst].cnt;
    return (c->off[MR_CLS_GHOST][l + 1] - c->off[MR_CLS_GHOST][l] + c->off[MR_CLS_LEAF][l + 1] -
            c->off[MR_CLS_LEAF][l] + TC - 1) / TC;
  });
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int tt = blockIdx.x; tt < tiles; tt += gridDim.x) {  // uniform over the block
    const int b = mr_group_find(pre, ngrp, tt);
    mr_inst_use(si, have, IB, b);
    const Geo& g = si.g;
    const MeshDev& Bm = si.mesh[dst];
    void* LF = si.fscratch;
    const int level = g.Jmin + kl;
    const int gb = Bm.cnt->off[MR_CLS_GHOST][level], ge = Bm.cnt->off[MR_CLS_GHOST][level + 1];
    const int lb = Bm.cnt->off[MR_CLS_LEAF][level], le = Bm.cnt->off[MR_CLS_LEAF][level + 1];
    const int ng = ge - gb, total = ng + (le - lb);
    const int t = (tt - pre[b]) * TC + tx;
    bool active = t < total;
    uint32_t code = 0;
    St* out = nullptr;
    size_t ostride = 0;
    if (active) {
      if (t < ng) {
        const int i = gb + t;
        code = Bm.code[MR_CLS_GHOST][i];
        out = (St*)Bm.GF + i;
        ostride = g.cap[2];
      } else {
        const int i = lb + (t - ng);
        active = Bm.src[i] < 0;  // a leaf carried over keeps its transferred values
        code = Bm.code[MR_CLS_LEAF][i];
        out = (St*)LF + i;
        ostride = g.cap[0];
      }
    }
    __syncthreads();  // the previous tile's readers of sent are done
    if (active) {
      int pc[3] = {0, 0, 0};
      mr_decode_d<D>(g, level - 1, code >> D, pc);
      for (int e = ty; e < B::N; e += 8) sent[e][tx] = wide_stencil_entry<D, S>(g, Bm, level - 1, pc, e);
    }
    __syncthreads();
    if (!active) continue;
    bool ok = true;
    for (int k = 0; k < B::N; ++k) ok = ok && sent[k][tx] != MR_MAP_NONE;
    if (!ok) {
      if (ty == 0) mr_set_err(Bm.cnt, MR_DERR_INTERNAL);
      continue;
    }
    const int ci = (int)(code & ((1u << D) - 1u));
    for (int p = ty; p < g.Q; p += 8) {
      C v[B::N];
      for (int k = 0; k < B::N; ++k) v[k] = ld_c<C>(mr_resolve<St>(g, Bm, LF, sent[k][tx]), p);
      out[(size_t)p * ostride] = mr_from_d<St>((double)wide_predict<D, S, C, false>(v, ci, g.cross_sign));
    }
  }
}

// ------------------------------------------------------------------ uniform-level reconstruction
// Conserved moments on the uniform level `level`: values of the complete
// tree where present, the prediction of half-width s of the level above
// otherwise (the prediction is linear, so it acts on the moments).
template <int D, int S, int F>
__global__ void __launch_bounds__(256) k_project_dense_w(Geo g, MeshDev Bm, const void* __restrict__ LF, int level,
                                                         const double* __restrict__ prev, double* cur) {
  using St = typename FormT<F>::S;
  using B = WBox<D, S>;
  const int n0 = g.n[level][0], n1 = g.n[level][1];
  const long long N = (long long)n0 * n1 * g.n[level][2];
  const int p0 = level > g.Jmin ? g.n[level - 1][0] : 1, p1 = level > g.Jmin ? g.n[level - 1][1] : 1;
  const long long PN = level > g.Jmin ? (long long)p0 * p1 * g.n[level - 1][2] : 1;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x) {
    const int c[3] = {(int)(r % n0), (int)((r / n0) % n1), (int)(r / ((long long)n0 * n1))};
    const int32_t e = Bm.map[g.base[level] + mr_encode_d<D>(g, level, c)];
    if (e != MR_MAP_NONE && (((uint32_t)e) >> 30) <= MR_CLS_INT) {
      const ValPtr<St> v = mr_resolve<St>(g, Bm, LF, e);
      for (int k = 0; k < g.ncons; ++k) {
        double acc = 0.0;
        for (int p = 0; p < g.Q; ++p) acc += g.consw[k][p] * (mr_ld(v, p) + (FormT<F>::offs ? g.off[p] : 0.0));
        cur[k * N + r] = acc;
      }
    } else if (level > g.Jmin) {
      int ci = 0;
      for (int a = 0; a < D; ++a) ci |= (c[a] & 1) << a;
      for (int k = 0; k < g.ncons; ++k) {
        double v[B::N];
        for (int q = 0; q < B::N; ++q) {
          int s[3] = {(c[0] >> 1) + q % B::W1 - S, D >= 2 ? (c[1] >> 1) + (q / B::W1) % B::W1 - S : 0,
                      D == 3 ? (c[2] >> 1) + q / (B::W1 * B::W1) - S : 0};
          mr_nbr_stencil_d<D>(g, level - 1, s);
          v[q] = prev[k * PN + ((long long)s[2] * p1 + s[1]) * p0 + s[0]];
        }
        cur[k * N + r] = wide_predict<D, S, double, false>(v, ci, g.cross_sign);
      }
    } else {
      mr_set_err(Bm.cnt, MR_DERR_INTERNAL);
    }
  }
}

// ------------------------------------------------------------------ critical-case details
// The details of the children of every refined cell that a leaf of its own
// level can reach with its window (W = 2s cells along an axis, or the
// (2W+1)^2 block of a lattice with diagonal velocities), for every
// population: det[(child * Q + p) * cap_int + i] = child value minus its
// prediction from the refined cell's (2s+1)^d stencil, in the form's
// arithmetic, the operations the transport would perform.  The transport
// then reads them for every refined cell of its window instead of
// predicting the children again for each leaf and population.
template <int D, int S, int F>
__global__ void __launch_bounds__(128) k_edge_details_w(const InstDev* __restrict__ IB, int ngrp, int dst) {
  using St = typename FormT<F>::S;
  using C = typename FormT<F>::C;
  using B = WBox<D, S>;
  constexpr int W = 2 * S, NW = 2 * W + 1;
  extern __shared__ int pre[];
  __shared__ InstDev si;
  int have = -1;
  mr_inst_prefetch(si, have, IB, ngrp);
  mr_grid_dep();
  const int tiles =
      mr_group_prefix(pre, ngrp, [&](int b) { return (IB[b].mesh[dst].cnt->total[MR_CLS_INT] + 127) / 128; });
  for (int tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
    const int b = mr_group_find(pre, ngrp, tt);
    mr_inst_use(si, have, IB, b);
    const Geo& g = si.g;
    const MeshDev& Bm = si.mesh[dst];
    const int i = (tt - pre[b]) * 128 + threadIdx.x;
    if (i >= Bm.cnt->total[MR_CLS_INT]) continue;
    const int l = Bm.lvl[MR_CLS_INT][i];
    const uint32_t code = Bm.code[MR_CLS_INT][i];
    int c[3] = {0, 0, 0};
    mr_decode_d<D>(g, l, code, c);
    // does a leaf of level l reach it?
    const bool block = D == 2 && g.diag;
    const int nw = block ? NW * NW : D * 2 * W;
    bool need = false;
    for (int w = 0; w < nw && !need; ++w) {
      int nb[3] = {c[0], c[1], c[2]};
      if (block) {
        if (w == NW * W + W) continue;
        nb[0] += w % NW - W;
        nb[1] += w / NW - W;
      } else {
        const int axis = w / (2 * W), o = w % (2 * W);
        nb[axis] += o < W ? o - W : o - W + 1;
      }
      if (!mr_nbr_mesh_d<D>(g, l, nb)) continue;
      const int32_t e = Bm.map[g.base[l] + mr_encode_d<D>(g, l, nb)];
      need = e != MR_MAP_NONE && (((uint32_t)e) >> 30) == MR_CLS_LEAF;
    }
    if (!need) continue;
    int32_t st[B::N], ce[1 << D];
    bool ok = wide_stencil<D, S>(g, Bm, l, c, st);
    for (int ci = 0; ci < (1 << D); ++ci) {
      ce[ci] = Bm.map[g.base[l + 1] + ((code << D) | (uint32_t)ci)];
      ok = ok && ce[ci] != MR_MAP_NONE;
    }
    if (!ok) {
      mr_set_err(Bm.cnt, MR_DERR_INTERNAL);
      continue;
    }
    const St* LFin = (const St*)si.fscratch;
    C* det = (C*)si.det;
    const size_t cap1 = g.cap[1];
    for (int p = 0; p < g.Q; ++p) {
      C v[B::N];
      for (int kk = 0; kk < B::N; ++kk) v[kk] = ld_c<C>(mr_resolve<St>(g, Bm, LFin, st[kk]), p);
      for (int ci = 0; ci < (1 << D); ++ci)
        det[((size_t)ci * g.Q + p) * cap1 + i] =
            ld_c<C>(mr_resolve<St>(g, Bm, LFin, ce[ci]), p) - wide_predict<D, S, C, false>(v, ci, g.cross_sign);
    }
  }
}

// ------------------------------------------------------------------ transport + collision
#define MR_WOUT ((int32_t)0xC0000000)  // window cell outside a non-periodic domain

template <class C>
__device__ __forceinline__ const C* wide_tab(const InstDev& si);
template <>
__device__ __forceinline__ const double* wide_tab<double>(const InstDev& si) { return si.Ws; }
template <>
__device__ __forceinline__ const float* wide_tab<float>(const InstDev& si) { return si.Wsf; }

// Weight of the level-l1 cell at position 2k + rel along axis a in the
// incoming-minus-outgoing finest values of the level-(l1 - 1) leaf k, for
// the velocity sign s (the corner cells of a diagonal velocity): s > 0:
// R_{2k-1} - R_{2k+1}, s < 0: L_{2k+2} - L_{2k}; the upwind term is absent at
// a non-periodic face (that cell is outside the domain).
template <class C>
__device__ __forceinline__ C wide_corner_weight(const Geo& g, const C* __restrict__ Wt, int l1, int a, int k, int rel,
                                                int s, int W) {
  const int per = g.periodic[a], N1 = g.n[l1][a], N = g.n[l1 - 1][a];
  const int tab = s > 0 ? 2 : 3;
  const int ru = s > 0 ? -1 : 2, ro = s > 0 ? 1 : 0;
  const int du = rel - ru, dd = rel - ro;
  C w = (C)0;
  if ((per || (s > 0 ? k > 0 : k < N - 1)) && du >= -W && du <= W)
    w += Wt[MR_WWIDX(l1, a, mr_slot_w(2 * k + ru, N1, per, W), tab, W) + du + W];
  if (dd >= -W && dd <= W) w -= Wt[MR_WWIDX(l1, a, mr_slot_w(2 * k + ro, N1, per, W), tab, W) + dd + W];
  return w;
}

// One thread per leaf.  Along each axis a the
// populations moving along a take the flattened weights of the leaf's slot
// over its row k - W .. k + W (W = 2s), the boundary value of a
// non-periodic face they enter through, and for every refined cell of the
// window the details of its children through the level-(j+1) edge weights:
// for a velocity +1 the finest cell upwind of the leaf is the right edge of
// level-(j+1) cell 2k - 1 and the leaf's last finest cell the right edge of
// 2k + 1; for -1 the left edges of 2k + 2 and 2k.  A child's detail is
// averaged over the 2^{d-1} children on the row (their transverse sum is
// what the row-collapsed reconstruction sees).
//
// Diagonal velocities (D2Q9): the sum over E minus the sum over A is the
// two axis strips (above) plus four single finest cells: + the one
// diagonally upwind of the leaf, + the leaf's own downwind corner cell, -
// the two that mix the two.  With the tensor-product prediction each is the
// product of two one-dimensional reconstructions, so together they are the
// product of the two axes' in-minus-out weights applied to the (2W+1)^2
// block of level-j values, plus, for every refined cell of the block, its
// children's details through the products of the level-(j+1) weights.  At
// a corner of a non-periodic domain the outside cells take the boundary
// value of the face crossed first along x, so the four cells leave minus
// the value of the y face.
template <int SC, int S, int F>
__global__ void __launch_bounds__(128) k_stream_collide_w(const InstDev* __restrict__ IB, int ngrp, int dst,
                                                          int do_stream, int do_collide, int count) {
  using Sc = Scheme<SC>;
  using St = typename FormT<F>::S;
  using C = typename FormT<F>::C;
  using B = WBox<Sc::D, S>;
  constexpr bool OFFS = FormT<F>::offs;
  constexpr int D = Sc::D, Q = Sc::Q, W = 2 * S, NW = 2 * W + 1;
  extern __shared__ int pre[];
  __shared__ InstDev si;
  int have = -1;
  mr_inst_prefetch(si, have, IB, ngrp);
  mr_grid_dep();
  const int tiles =
      mr_group_prefix(pre, ngrp, [&](int b) { return (IB[b].mesh[dst].cnt->total[MR_CLS_LEAF] + 127) / 128; });
  for (int tt = blockIdx.x; tt < tiles; tt += gridDim.x) {
    const int b = mr_group_find(pre, ngrp, tt);
    mr_inst_use(si, have, IB, b);
    const Geo& g = si.g;
    const MeshDev& Bm = si.mesh[dst];
    const St* __restrict__ LFin = (const St*)si.fscratch;
    St* __restrict__ LFout = (St*)si.fstate;
    const C* __restrict__ Wt = wide_tab<C>(si);
    const int i = (tt - pre[b]) * 128 + threadIdx.x;
    if (count && tt == pre[b] && threadIdx.x == 0) {
      Bm.cnt->leaf_updates += Bm.cnt->total[MR_CLS_LEAF];
      Bm.cnt->steps += 1;
    }
    if (i >= Bm.cnt->total[MR_CLS_LEAF]) continue;
    const int l = Bm.lvl[MR_CLS_LEAF][i];
    const uint32_t code = Bm.code[MR_CLS_LEAF][i];
    const C* offv = mr_offv<C>(g);
    C fs[Q], out[Q];
    for (int p = 0; p < Q; ++p) {
      const ValPtr<St> me{LFin + i, g.cap[0]};
      fs[p] = ld_off<F>(me, p, offv);
      out[p] = fs[p];
    }
    if (do_stream) {
      int xc[3] = {0, 0, 0};
      mr_decode_d<D>(g, l, code, xc);
      const C scale = (C)__longlong_as_double((long long)(1023 + l - g.J) << 52);  // 2^{l-J}, exact
#pragma unroll 1
      for (int a = 0; a < D; ++a) {
        const int k = xc[a], N = g.n[l][a], per = g.periodic[a];
        const int slot = mr_slot_w(k, N, per, W);
        const C* wP = Wt + MR_WWIDX(l, a, slot, 0, W);
        const C* wM = Wt + MR_WWIDX(l, a, slot, 1, W);
        const bool lo = !per && k == 0, hi = !per && k == N - 1;
        int32_t ent[NW];
        for (int o = 0; o < NW; ++o) {
          ent[o] = MR_WOUT;
          if (o == W) continue;
          int nb[3] = {xc[0], xc[1], xc[2]};
          nb[a] += o - W;
          if (!mr_nbr_mesh_d<D>(g, l, nb)) continue;
          const int32_t e = Bm.map[g.base[l] + mr_encode_d<D>(g, l, nb)];
          if (e == MR_MAP_NONE)
            mr_set_err(Bm.cnt, MR_DERR_INTERNAL);
          else
            ent[o] = e;
        }
        for (int p = 0; p < Q; ++p) {
          const int sgn = eta_of<Sc>(p, a);
          if (sgn == 0) continue;
          const C* w = sgn > 0 ? wP : wM;
          C acc = w[W] * fs[p];
          for (int o = 0; o < NW; ++o)
            if (ent[o] != MR_WOUT) acc += w[o] * ld_off<F>(mr_resolve<St>(g, Bm, LFin, ent[o]), p, offv);
          if (sgn > 0 && lo) acc += bc_value<C>(g, g.bc[2 * a], fs, p, Sc::opp(p));
          if (sgn < 0 && hi) acc += bc_value<C>(g, g.bc[2 * a + 1], fs, p, Sc::opp(p));
          out[p] += scale * acc;
        }
        // the critical case: refined cells of the window, their children's
        // details from the pre-pass (k_edge_details_w)
        const C* __restrict__ det = (const C*)si.det;
        const size_t cap1 = g.cap[1];
        for (int o = 0; o < NW; ++o) {
          if (ent[o] == MR_WOUT || (((uint32_t)ent[o]) >> 30) != MR_CLS_INT) continue;
          const int dlt = o - W;
          const uint32_t ridx = (uint32_t)ent[o] & 0x3FFFFFFFu;
          const int N1 = g.n[l + 1][a];
          for (int p = 0; p < Q; ++p) {
            const int sgn = eta_of<Sc>(p, a);
            if (sgn == 0) continue;
            const int rE = sgn > 0 ? -1 : 2, rA = sgn > 0 ? 1 : 0;  // edge cells, relative to 2k
            const int tab = sgn > 0 ? 2 : 3;
            const bool eIn = per || (sgn > 0 ? k > 0 : k < N - 1);
            const C* wE = eIn ? Wt + MR_WWIDX(l + 1, a, mr_slot_w(2 * k + rE, N1, per, W), tab, W) : nullptr;
            const C* wA = Wt + MR_WWIDX(l + 1, a, mr_slot_w(2 * k + rA, N1, per, W), tab, W);
            C corr = (C)0;
            for (int ci = 0; ci < (1 << D); ++ci) {
              const int cx = 2 * dlt + ((ci >> a) & 1);
              const int oE = cx - rE, oA = cx - rA;
              C wgt = (C)0;
              if (wE && oE >= -W && oE <= W) wgt += wE[oE + W];
              if (oA >= -W && oA <= W) wgt -= wA[oA + W];
              if (wgt == (C)0) continue;
              corr += wgt * det[((size_t)ci * Q + p) * cap1 + ridx];
            }
            out[p] += scale * (corr * ((C)1 / (C)(1 << (D - 1))));
          }
        }
      }
      if constexpr (Sc::DIAG) {
        using B2 = WBox<2, S>;
        constexpr int P0 = Sc::DIAG0;
        const int x = xc[0], y = xc[1], Nx = g.n[l][0], Ny = g.n[l][1];
        const int slx = mr_slot_w(x, Nx, g.periodic[0], W), sly = mr_slot_w(y, Ny, g.periodic[1], W);
        const C* wx[2] = {Wt + MR_WWIDX(l, 0, slx, 0, W), Wt + MR_WWIDX(l, 0, slx, 1, W)};
        const C* wy[2] = {Wt + MR_WWIDX(l, 1, sly, 0, W), Wt + MR_WWIDX(l, 1, sly, 1, W)};
        C acc[4] = {(C)0, (C)0, (C)0, (C)0};
        for (int bb = 0; bb < NW; ++bb) {
          const C wy0 = wy[0][bb], wy1 = wy[1][bb];
          if (wy0 == (C)0 && wy1 == (C)0) continue;  // zero row: adds nothing
          for (int aa = 0; aa < NW; ++aa) {
            const C wx0 = wx[0][aa], wx1 = wx[1][aa];
            if (wx0 == (C)0 && wx1 == (C)0) continue;
            const bool self = aa == W && bb == W;
            int32_t e = 0;
            if (!self) {
              int nb[3] = {x + aa - W, y + bb - W, 0};
              if (!mr_nbr_mesh_d<2>(g, l, nb)) continue;  // outside a non-periodic domain: zero weight
              e = Bm.map[g.base[l] + mr_encode_d<2>(g, l, nb)];
              if (e == MR_MAP_NONE) {
                mr_set_err(Bm.cnt, MR_DERR_INTERNAL);
                continue;
              }
            }
            const ValPtr<St> vp = mr_resolve<St>(g, Bm, LFin, e);
            for (int t = 0; t < 4; ++t) {
              const int p = P0 + t;
              const C wab = (Sc::eta(p, 0) > 0 ? wx0 : wx1) * (Sc::eta(p, 1) > 0 ? wy0 : wy1);
              if (wab == (C)0) continue;
              acc[t] += wab * (self ? fs[p] : ld_off<F>(vp, p, offv));
            }
          }
        }
        // refined cells of the block: their children's details
        if (l < g.J) {
          for (int bb = 0; bb < NW; ++bb)
            for (int aa = 0; aa < NW; ++aa) {
              if (aa == W && bb == W) continue;
              C wcx[2][2], wcy[2][2];  // [sign index][child offset]
              bool any = false;
              for (int sg = 0; sg < 2; ++sg)
                for (int o = 0; o < 2; ++o) {
                  wcx[sg][o] = wide_corner_weight<C>(g, Wt, l + 1, 0, x, 2 * (aa - W) + o, sg == 0 ? 1 : -1, W);
                  wcy[sg][o] = wide_corner_weight<C>(g, Wt, l + 1, 1, y, 2 * (bb - W) + o, sg == 0 ? 1 : -1, W);
                  any = any || wcx[sg][o] != (C)0;
                }
              if (!any) continue;
              int nb[3] = {x + aa - W, y + bb - W, 0};
              if (!mr_nbr_mesh_d<2>(g, l, nb)) continue;
              const int32_t e = Bm.map[g.base[l] + mr_encode_d<2>(g, l, nb)];
              if (e == MR_MAP_NONE || (((uint32_t)e) >> 30) != MR_CLS_INT) continue;
              const uint32_t ridx = (uint32_t)e & 0x3FFFFFFFu;  // its children's details: det (pre-pass)
              const C* __restrict__ det = (const C*)si.det;
              const size_t cap1 = g.cap[1];
              for (int t = 0; t < 4; ++t) {
                const int p = P0 + t;
                const int ix = Sc::eta(p, 0) > 0 ? 0 : 1, iy = Sc::eta(p, 1) > 0 ? 0 : 1;
                C corr = (C)0;
                for (int ci = 0; ci < 4; ++ci) {
                  const C w = wcx[ix][ci & 1] * wcy[iy][ci >> 1];
                  if (w == (C)0) continue;
                  corr += w * det[((size_t)ci * Q + p) * cap1 + ridx];
                }
                acc[t] += corr;
              }
            }
        }
        const C scale2 = scale * scale;
        for (int t = 0; t < 4; ++t) {
          const int p = P0 + t;
          const int sx = Sc::eta(p, 0), sy = Sc::eta(p, 1);
          const bool outx = !g.periodic[0] && (sx > 0 ? x == 0 : x == Nx - 1);
          const bool outy = !g.periodic[1] && (sy > 0 ? y == 0 : y == Ny - 1);
          if (outx && outy) acc[t] -= bc_value<C>(g, g.bc[sy > 0 ? 2 : 3], fs, p, Sc::opp(p));
          out[p] += scale2 * acc[t];
        }
      }
    }
    if (do_collide) {
      Sc::template collide<C>(g, out);
      if constexpr (Sc::DIAG) {
        if (g.obstacle) {
          const double phi = obstacle_fraction(g, l, code);
          if (phi > 0.0)
            for (int p = 0; p < Q; ++p) out[p] = (C)phi * MR_K(C, g, feq0[p]) + ((C)1 - (C)phi) * out[p];
        }
      }
    }
    bool finite = true;
    for (int p = 0; p < Q; ++p) {
      finite = finite && is_finite_bits(out[p]);
      if constexpr (OFFS)
        LFout[(size_t)p * g.cap[0] + i] = mr_from_f<St>((float)(out[p] - offv[p]));
      else
        LFout[(size_t)p * g.cap[0] + i] = (St)out[p];
    }
    if (!finite) mr_set_err(Bm.cnt, MR_DERR_NONFINITE);
  }
}

// ------------------------------------------------------------------ launchers
template <int D, int S, int F>
void launch_details_w(const Group& G, int cur, cudaStream_t st) {
  constexpr int TC = WTile<D, S>::TC;
  mr_launch_pdl(k_details_w<D, S, F>, mr_tile_grid(G, G.capI, TC, G.bps[MR_PH_DETAILS]), dim3(TC, 8), mr_pre_bytes(G),
                st, G.dev, G.n, cur);
}
template <int D, int S, int F>
void launch_predict_w(const Group& G, int dst, int kl, cudaStream_t st) {
  constexpr int TC = WTile<D, S>::TC;
  mr_launch_pdl(k_predict_level_w<D, S, F>, mr_tile_grid(G, 2 * G.pred_cells[kl], TC, G.bps[MR_PH_PREDICT]),
                dim3(TC, 8), mr_pre_bytes(G), st, G.dev, G.n, dst, kl);
}
template <int D, int S, int F>
void launch_edge_w(const Group& G, int dst, cudaStream_t st) {
  mr_launch_pdl(k_edge_details_w<D, S, F>, mr_tile_grid(G, G.capI, 128, G.bps[MR_PH_STREAM]), 128, mr_pre_bytes(G), st,
                G.dev, G.n, dst);
}
template <int SC, int S, int F>
void launch_stream_w(const Group& G, int dst, int ds, int dc, int count, cudaStream_t st) {
  mr_launch_pdl(k_stream_collide_w<SC, S, F>, mr_tile_grid(G, G.capL, 128, G.bps[MR_PH_STREAM]), 128, mr_pre_bytes(G), st, G.dev, G.n,
                dst, ds, dc, count);
}
template <int D, int S, int F>
void launch_dense_w(const Geo& g, const MeshDev& B, const void* LF, int level, const double* prev, double* cur,
                    cudaStream_t st, int grid) {
  k_project_dense_w<D, S, F><<<grid, 256, 0, st>>>(g, B, LF, level, prev, cur);
}

}  // namespace

// form, then half-width
#define MR_W_FORMS(FN, FORM, PRE, ...)                                          \
  switch (FORM) {                                                               \
    case MR_FORM_F64: FN<PRE, MR_FORM_F64>(__VA_ARGS__); break;                 \
    case MR_FORM_F32: FN<PRE, MR_FORM_F32>(__VA_ARGS__); break;                 \
    case MR_FORM_F32_F16: FN<PRE, MR_FORM_F32_F16>(__VA_ARGS__); break;         \
    case MR_FORM_F32_BF16: FN<PRE, MR_FORM_F32_BF16>(__VA_ARGS__); break;       \
  }
#define MR_W_S(FN, FORM, S_, A1, ...)                                   \
  do {                                                                  \
    if ((S_) == 2) {                                                    \
      MR_W_FORMS(FN, FORM, MR_W_PAIR(A1, 2), __VA_ARGS__);              \
    } else {                                                            \
      MR_W_FORMS(FN, FORM, MR_W_PAIR(A1, 3), __VA_ARGS__);              \
    }                                                                   \
  } while (0)
#define MR_W_PAIR(a, b) a, b

void mr_launch_details_w(const Group& G, int cur, cudaStream_t st) {
  if (G.d == 1) MR_W_S(launch_details_w, G.form, G.s, 1, G, cur, st);
  else if (G.d == 2) MR_W_S(launch_details_w, G.form, G.s, 2, G, cur, st);
  else MR_W_S(launch_details_w, G.form, G.s, 3, G, cur, st);
}

void mr_launch_predict_level_w(const Group& G, int dst, int kl, cudaStream_t st) {
  if (G.d == 1) MR_W_S(launch_predict_w, G.form, G.s, 1, G, dst, kl, st);
  else if (G.d == 2) MR_W_S(launch_predict_w, G.form, G.s, 2, G, dst, kl, st);
  else MR_W_S(launch_predict_w, G.form, G.s, 3, G, dst, kl, st);
}

void mr_launch_edge_details_w(const Group& G, int dst, cudaStream_t st) {
  if (G.d == 1) MR_W_S(launch_edge_w, G.form, G.s, 1, G, dst, st);
  else if (G.d == 2) MR_W_S(launch_edge_w, G.form, G.s, 2, G, dst, st);
  else MR_W_S(launch_edge_w, G.form, G.s, 3, G, dst, st);
}

void mr_launch_stream_collide_w(const Group& G, int dst, int do_stream, int do_collide, cudaStream_t st, int count) {
  switch (G.scheme) {
    case 0: MR_W_S(launch_stream_w, G.form, G.s, 0, G, dst, do_stream, do_collide, count, st); break;
    case 1: MR_W_S(launch_stream_w, G.form, G.s, 1, G, dst, do_stream, do_collide, count, st); break;
    case 2: MR_W_S(launch_stream_w, G.form, G.s, 2, G, dst, do_stream, do_collide, count, st); break;
    case 3: MR_W_S(launch_stream_w, G.form, G.s, 3, G, dst, do_stream, do_collide, count, st); break;
    case 4: MR_W_S(launch_stream_w, G.form, G.s, 4, G, dst, do_stream, do_collide, count, st); break;
    case 5: MR_W_S(launch_stream_w, G.form, G.s, 5, G, dst, do_stream, do_collide, count, st); break;
    default: break;
  }
}

void mr_launch_grade_w(const Group& G, cudaStream_t st) {
  if (!G.grade) return;
  const int grid = mr_tile_grid(G, (long long)G.chunks * MR_DENSE_ALIGN, 256, G.bps[MR_PH_FLAGS]);
  const size_t sm = mr_pre_bytes(G);
  if (G.d == 1) {
    if (G.s == 2) mr_launch_pdl(k_grade_w<1, 2>, grid, 256, sm, st, G.dev, G.n);
    else mr_launch_pdl(k_grade_w<1, 3>, grid, 256, sm, st, G.dev, G.n);
  } else if (G.d == 2) {
    if (G.s == 2) mr_launch_pdl(k_grade_w<2, 2>, grid, 256, sm, st, G.dev, G.n);
    else mr_launch_pdl(k_grade_w<2, 3>, grid, 256, sm, st, G.dev, G.n);
  } else {
    if (G.s == 2) mr_launch_pdl(k_grade_w<3, 2>, grid, 256, sm, st, G.dev, G.n);
    else mr_launch_pdl(k_grade_w<3, 3>, grid, 256, sm, st, G.dev, G.n);
  }
}

void mr_launch_mark_ghosts_w(const Group& G, cudaStream_t st) {
  const int grid = mr_chunk_blocks_grid(G);
  if (G.d == 1) {
    if (G.s == 2) mr_launch_pdl(k_mark_ghosts_w<1, 2>, grid, 256, 0, st, G.dev, G.chunk_pre, G.n, G.chunks);
    else mr_launch_pdl(k_mark_ghosts_w<1, 3>, grid, 256, 0, st, G.dev, G.chunk_pre, G.n, G.chunks);
  } else if (G.d == 2) {
    if (G.s == 2) mr_launch_pdl(k_mark_ghosts_w<2, 2>, grid, 256, 0, st, G.dev, G.chunk_pre, G.n, G.chunks);
    else mr_launch_pdl(k_mark_ghosts_w<2, 3>, grid, 256, 0, st, G.dev, G.chunk_pre, G.n, G.chunks);
  } else {
    if (G.s == 2) mr_launch_pdl(k_mark_ghosts_w<3, 2>, grid, 256, 0, st, G.dev, G.chunk_pre, G.n, G.chunks);
    else mr_launch_pdl(k_mark_ghosts_w<3, 3>, grid, 256, 0, st, G.dev, G.chunk_pre, G.n, G.chunks);
  }
}

void mr_launch_project_dense_w(const Geo& g, const MeshDev& B, const void* LF, int level, const double* prev,
                               double* cur, cudaStream_t st, int grid) {
  if (g.d == 1) MR_W_S(launch_dense_w, g.form, g.s_pred, 1, g, B, LF, level, prev, cur, st, grid);
  else if (g.d == 2) MR_W_S(launch_dense_w, g.form, g.s_pred, 2, g, B, LF, level, prev, cur, st, grid);
  else MR_W_S(launch_dense_w, g.form, g.s_pred, 3, g, B, LF, level, prev, cur, st, grid);
}

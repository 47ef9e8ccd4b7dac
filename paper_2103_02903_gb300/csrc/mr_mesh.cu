// Mesh adaptation on the GPU (Sec. 4.3, 4.4, 5.1): the threshold operator
// T_eps with its tree closure, the enlargement H_eps, the grading G, the
// classification of every cell of the new tree, the marking of the ghost
// cells whose reconstructed values the transport reads, and the compaction
// of leaves / internal cells / ghosts into per-level sorted Morton-key
// arrays with a dense per-level index map.
//
// The tree is held as one "refined" flag per cell of levels J_min..J-1: a
// cell belongs to R(Lambda) iff it is on level J_min or its parent is
// refined.  Every mark is an idempotent byte OR, so races between threads
// are benign; the closure under ancestors and the grading cascade are
// walked by the thread that first sets a flag, which makes each of them a
// single kernel whatever the number of levels.
//
// The dense arrays are visited chunk by chunk (1024 cells of one level), and
// only the chunks a writer touched: every flag, class or ghost mark also
// stores 1 into the chunk's activity byte (act; acth for the H flags that
// seed the grading), a refined cell touching the chunk of its children too,
// so that a chunk never touched keeps all its flag and class bytes at 0 and
// is skipped.  The compaction clears the bytes of the chunks it visits, and
// rewrites a chunk of the new index map only if it holds entries now or did
// in the mesh last written there (mact).
#include "mr_common.cuh"

namespace {

__device__ __forceinline__ double level_eps(const Geo& g, int l) { return ldexp(g.eps, g.d * (l - g.J)); }

// A cell (level L < J, code c) newly refined (H or G): its own chunk and the
// chunk of its children (all 2^D of them in one chunk) hold cells of the new
// tree; an H cell also seeds the grading from its chunk.
template <int D>
__device__ __forceinline__ void touch_refined(const InstDev& si, int L, uint32_t c, bool seed) {
  const uint32_t gi = si.g.base[L] + c;
  mr_touch(si.act, gi);
  mr_touch(si.act, si.g.base[L + 1] + (c << D));
  if (seed) mr_touch(si.acth, gi);
}

// ---------------------------------------------------------------- T_eps
// Tiled step kernels over the internal cells of the current mesh: a tile is
// 256 cells of one instance.
#define MR_INT_TILES_BEGIN(IB, N, CUR, G_, A_, I_)                                              \
  extern __shared__ int pre[];                                                                \
  __shared__ InstDev si;                                                                      \
  int have = -1;                                                                              \
  mr_inst_prefetch(si, have, IB, N);                                                          \
  mr_grid_dep();                                                                              \
  const int tiles =                                                                           \
      mr_group_prefix(pre, N, [&](int b) { return (IB[b].mesh[CUR].cnt->total[MR_CLS_INT] + 255) / 256; }); \
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {                                        \
    const int b = mr_group_find(pre, N, t);                                                   \
    mr_inst_use(si, have, IB, b);                                                             \
    const Geo& G_ = si.g;                                                                     \
    const MeshDev& A_ = si.mesh[CUR];                                                         \
    const int I_ = (t - pre[b]) * 256 + threadIdx.x;                                          \
    if (I_ >= A_.cnt->total[MR_CLS_INT]) continue;
#define MR_INT_TILES_END }

template <int D>
__global__ void __launch_bounds__(256) k_flags_T(const InstDev* __restrict__ IB, int n, int cur) {
  MR_INT_TILES_BEGIN(IB, n, cur, g, A, i)
    uint8_t* flags = si.flags;
    const int L = A.lvl[MR_CLS_INT][i];
    if (!(A.G[i] >= level_eps(g, L + 1))) continue;
    int l = L;
    uint32_t c = A.code[MR_CLS_INT][i];
    for (;;) {
      // a plain load first: most ancestors are already marked
      if (flags[g.base[l] + c] & MR_F_T) break;
      uint32_t old = mr_atomic_or_byte(flags, g.base[l] + c, MR_F_T);
      if (!old) mr_touch(si.act, g.base[l] + c);
      if ((old & MR_F_T) || l == g.Jmin) break;
      --l;
      c >>= D;
    }
  MR_INT_TILES_END
}

// ---------------------------------------------------------------- H_eps
template <int D>
__global__ void __launch_bounds__(256) k_flags_H(const InstDev* __restrict__ IB, int n, int cur) {
  MR_INT_TILES_BEGIN(IB, n, cur, g, A, i)
    uint8_t* flags = si.flags;
    const int L = A.lvl[MR_CLS_INT][i];
    const uint32_t code = A.code[MR_CLS_INT][i];
    if (!(flags[g.base[L] + code] & MR_F_T)) continue;
    mr_atomic_or_byte(flags, g.base[L] + code, MR_F_H);
    touch_refined<D>(si, L, code, true);
    int c0[3] = {0, 0, 0};
    mr_decode_d<D>(g, L, code, c0);
    // neighbour rule (Eq. AdditionNeigh) on the children, which are the
    // cells of R(T_eps(Lambda)) on level L+1
    for (int ci = 0; ci < (1 << D); ++ci) {
      for (int h = 0; h < g.q; ++h) {
        int nb[3] = {0, 0, 0};
        for (int a = 0; a < D; ++a) nb[a] = 2 * c0[a] + ((ci >> a) & 1) - g.eta[h][a];
        if (!mr_nbr_mesh_d<D>(g, L + 1, nb)) continue;
        for (int a = 0; a < D; ++a) nb[a] >>= 1;
        const uint32_t nc = mr_encode_d<D>(g, L, nb), gi = g.base[L] + nc;
        if (!(flags[gi] & MR_F_H) && !(mr_atomic_or_byte(flags, gi, MR_F_H) & MR_F_H))
          touch_refined<D>(si, L, nc, true);
      }
    }
    // refinement rule (Sec. 5.1): J_min < L+1 < J and group norm >= 2^{mu+d} eps_{L+1}
    if (L + 1 > g.Jmin && L + 1 < g.J && A.G[i] >= ldexp(level_eps(g, L + 1), g.mu_bar + D)) {
      for (int ci = 0; ci < (1 << D); ++ci)
        mr_atomic_or_byte(flags, g.base[L + 1] + ((code << D) | (uint32_t)ci), MR_F_H);
      touch_refined<D>(si, L + 1, code << D, true);  // the children share their chunks
    }
  MR_INT_TILES_END
}

// ---------------------------------------------------------------- grading
// Every refined cell p of level L >= J_min+1 needs the 3^d stencil of its
// children (the cells around p on level L) in the tree, i.e. the parents of
// those cells refined on level L-1.  The thread that newly refines a cell
// continues the cascade from it, depth first, towards J_min.  Each frame of
// the cascade first reads the flags of all its parents together (independent
// loads) and keeps a bit mask of those not refined yet; only those are then
// set one by one with the atomic OR.
template <int D>
__device__ __forceinline__ uint32_t grade_need(const Geo& g, const uint8_t* flags, int L, int x, int y) {
  uint32_t m = 0;
  const uint8_t* fl = flags + g.base[L - 1];
  if constexpr (D == 2) {
    MortonBox<1> bx;
    bx.init(g, L, x, y, true);
#pragma unroll
    for (int k = 0; k < 9; ++k)
      if (bx.in(k % 3, k / 3) && !(fl[bx.code(k % 3, k / 3)] & (MR_F_H | MR_F_G))) m |= 1u << k;
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int nx = x + k - 1, ny = 0;
      if (!mr_nbr_mesh(g, L, nx, ny)) continue;
      if (!(fl[mr_encode(g, L - 1, nx >> 1, 0)] & (MR_F_H | MR_F_G))) m |= 1u << k;
    }
  }
  return m;
}
// d = 3: the 27 neighbours of (x, y, z) on level L, their parents on L - 1
__device__ __forceinline__ uint32_t grade_need3(const Geo& g, const uint8_t* flags, int L, const int* c) {
  uint32_t m = 0;
  const uint8_t* fl = flags + g.base[L - 1];
  MortonBox3<1> bx;
  bx.init(g, L, c, true);
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const int i = k % 3, j = (k / 3) % 3, kk = k / 9;
    if (bx.inside(i, j, kk) && !(fl[bx.code(i, j, kk)] & (MR_F_H | MR_F_G))) m |= 1u << k;
  }
  return m;
}

template <int D>
__global__ void __launch_bounds__(256) k_grade(const InstDev* __restrict__ IB, int n) {
  // tiles of 256 cells strided over the grid (not one block per chunk):
  // refined cells cluster, and interleaving spreads their cascades
  extern __shared__ int pre[];
  __shared__ InstDev si;
  int have = -1;
  mr_inst_prefetch(si, have, IB, n);
  mr_grid_dep();  // after the copy of the descriptor, which no step kernel writes
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
    int sl[MR_MAXL], sx[MR_MAXL], sy[MR_MAXL], sz[MR_MAXL];
    uint32_t sm[MR_MAXL];
    int sp = 1;
    sl[0] = l0;
    {
      int c[3] = {0, 0, 0};
      mr_decode_d<D>(g, l0, c0, c);
      sx[0] = c[0];
      sy[0] = c[1];
      sz[0] = c[2];
      if constexpr (D == 3)
        sm[0] = grade_need3(g, flags, l0, c);
      else
        sm[0] = grade_need<D>(g, flags, l0, sx[0], sy[0]);
    }
    while (sp > 0) {
      const int t = sp - 1;
      if (sm[t] == 0u) {
        --sp;
        continue;
      }
      const int k = __ffs(sm[t]) - 1;
      sm[t] &= sm[t] - 1u;
      const int L = sl[t];
      int nb[3] = {sx[t] + (k % 3) - 1, D >= 2 ? sy[t] + (k / 3) % 3 - 1 : 0, D == 3 ? sz[t] + k / 9 - 1 : 0};
      mr_nbr_mesh_d<D>(g, L, nb);  // inside: only such cells enter the mask
      const int tl = L - 1;
      for (int a = 0; a < D; ++a) nb[a] >>= 1;
      const uint32_t nc = mr_encode_d<D>(g, tl, nb);
      const uint32_t old = mr_atomic_or_byte(flags, g.base[tl] + nc, MR_F_G);
      if (!(old & (MR_F_H | MR_F_G))) touch_refined<D>(si, tl, nc, false);
      if (!(old & (MR_F_H | MR_F_G)) && tl > g.Jmin && sp < MR_MAXL) {
        sl[sp] = tl;
        sx[sp] = nb[0];
        sy[sp] = nb[1];
        sz[sp] = nb[2];
        if constexpr (D == 3)
          sm[sp] = grade_need3(g, flags, tl, nb);
        else
          sm[sp] = grade_need<D>(g, flags, tl, nb[0], nb[1]);
        ++sp;
      }
    }
  }
}

// ---------------------------------------------------------------- classify
// One warp per touched chunk, grid-stride over the chunks of all instances:
// lane L classifies cells 32L .. 32L+31 of the chunk from their own flag
// bytes (two 16-byte loads) and their parents' (32 >> D consecutive bytes),
// and writes the 32 class bytes with two 16-byte stores.  A chunk of a level
// above J_min that nothing touched has no refined parent: its class bytes
// stay 0.
template <int D>
__global__ void __launch_bounds__(256) k_classify(const InstDev* __restrict__ IB,
                                                  const int* __restrict__ chunk_pre, int n, int nchunks) {
  mr_grid_dep();
  const int lane = threadIdx.x & 31;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < nchunks; t += nw) {
    int chunk;
    const InstDev& I = IB[mr_group_chunk_of(chunk_pre, n, t, chunk)];
    const Geo& g = I.g;
    const uint32_t c0 = (uint32_t)chunk * MR_DENSE_ALIGN;
    const int l = mr_level_of(g, c0);
    const bool top = l == g.Jmin;
    if (!top && !__shfl_sync(0xffffffffu, (int)I.act[chunk], 0)) continue;
    if (top && lane == 0) I.act[chunk] = 1;  // the counts and the scatter visit it
    const uint32_t first = c0 - g.base[l] + 32u * (uint32_t)lane, ncode = g.ncode[l];
    uint32_t fw[8] = {0, 0, 0, 0, 0, 0, 0, 0}, pw[4] = {0, 0, 0, 0};
    if (l < g.J) {
      const uint4* fp = (const uint4*)(I.flags + c0) + 2 * lane;
      const uint4 a = fp[0], b = fp[1];
      fw[0] = a.x; fw[1] = a.y; fw[2] = a.z; fw[3] = a.w;
      fw[4] = b.x; fw[5] = b.y; fw[6] = b.z; fw[7] = b.w;
    }
    if (!top) {
      const uint8_t* pp = I.flags + g.base[l - 1] + (first >> D);  // 32 >> D bytes, aligned to their size
      if constexpr (D == 1) {
        const uint4 a = *(const uint4*)pp;
        pw[0] = a.x; pw[1] = a.y; pw[2] = a.z; pw[3] = a.w;
      } else if constexpr (D == 2) {
        const uint2 a = *(const uint2*)pp;
        pw[0] = a.x; pw[1] = a.y;
      } else {
        pw[0] = *(const uint32_t*)pp;
      }
    }
    uint32_t ow[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      uint32_t o = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int j = 4 * w + k, pj = j >> D;
        const uint32_t pb = (pw[pj >> 2] >> (8 * (pj & 3))) & 0xFFu, fb = (fw[w] >> (8 * k)) & 0xFFu;
        const bool inR = top || (pb & (MR_F_H | MR_F_G));
        const uint32_t v = !inR || first + (uint32_t)j >= ncode ? 0u : ((fb & (MR_F_H | MR_F_G)) ? MR_C_INT : MR_C_LEAF);
        o |= v << (8 * k);
      }
      ow[w] = o;
    }
    uint4* cp = (uint4*)(I.cls + c0) + 2 * lane;
    cp[0] = make_uint4(ow[0], ow[1], ow[2], ow[3]);
    cp[1] = make_uint4(ow[4], ow[5], ow[6], ow[7]);
  }
}

__global__ void __launch_bounds__(256) k_full_mesh(Geo g, uint8_t* cls, uint8_t* act) {
  if (threadIdx.x == 0) act[blockIdx.x] = 1;
  MR_DENSE_CHUNK_BEGIN(g, blockIdx.x, l, c, gi)
    (void)c;
    cls[gi] = l == g.J ? MR_C_LEAF : MR_C_INT;
  MR_DENSE_CHUNK_END
}

// ---------------------------------------------------------------- ghosts
// The transport of a leaf on level l reads the reconstructed values of the
// cells at distance 1 and 2 along each axis on level l (the flattened
// window), and, for a lattice with diagonal velocities, the whole 5 x 5
// block around the leaf.  Those outside R(Lambda) are ghosts: predicted from
// level l-1, whose stencil cells outside R(Lambda) are ghosts in turn.
// The classes of a window (and of each stencil of the cascade) are read
// together first, as independent loads; only the cells still unmarked are
// then marked one by one with the atomic OR.
template <int D>
__device__ __forceinline__ uint32_t ghost_stencil_need(const Geo& g, const uint8_t* cls, int L, int x, int y) {
  uint32_t m = 0;
  const uint8_t* cl = cls + g.base[L];
  if constexpr (D == 2) {
    MortonBox<1> bx;
    bx.init(g, L, x, y);
#pragma unroll
    for (int k = 0; k < 9; ++k)
      if (bx.in(k % 3, k / 3) && !(cl[bx.code(k % 3, k / 3)] & (3u | MR_C_GHOST))) m |= 1u << k;
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int ax = x + k - 1, ay = 0;
      if (!mr_nbr_mesh(g, L, ax, ay)) continue;
      if (!(cl[mr_encode(g, L, ax, 0)] & (3u | MR_C_GHOST))) m |= 1u << k;
    }
  }
  return m;
}

// window cell w of a leaf at (x, y): the 5 x 5 block (w = 5 row + column)
// or the axis windows (w = 4 axis + k, offsets -2, -1, +1, +2)
__device__ __forceinline__ void ghost_window_cell(bool block, int w, int x, int y, int& nx, int& ny) {
  if (block) {
    nx = x + w % 5 - 2;
    ny = y + w / 5 - 2;
  } else {
    const int axis = w >> 2, k = w & 3;
    const int off = k < 2 ? k - 2 : k - 1;
    nx = x + (axis == 0 ? off : 0);
    ny = y + (axis == 1 ? off : 0);
  }
}

// d = 3: the 12 axis window cells of a leaf (4 per axis), each cell outside
// the tree marked with the cascade over the 27-cell stencils of its parents
__device__ __forceinline__ uint32_t ghost_need3(const Geo& g, const uint8_t* cls, int L, const int* c) {
  uint32_t m = 0;
  const uint8_t* cl = cls + g.base[L];
  MortonBox3<1> bx;
  bx.init(g, L, c);
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const int i = k % 3, j = (k / 3) % 3, kk = k / 9;
    if (bx.inside(i, j, kk) && !(cl[bx.code(i, j, kk)] & (3u | MR_C_GHOST))) m |= 1u << k;
  }
  return m;
}

// A cell of level L + 1 became a ghost: mark its parent's 3^D stencil
// (cell c of level L), cells outside the tree becoming ghosts, and so on
// towards J_min, depth first; only the thread that marks a cell first walks
// on from it, and only the thread that claims a stencil first walks it.
template <int D>
__device__ void ghost_cascade(const Geo& g, uint8_t* cls, uint8_t* act, int L0, const int* c0) {
  if (!mr_claim_stencil(cls, act, g.base[L0] + mr_encode_d<D>(g, L0, c0))) return;
  int sl[MR_MAXL], sc[MR_MAXL][3];
  uint32_t sm[MR_MAXL];
  sl[0] = L0;
  for (int a = 0; a < 3; ++a) sc[0][a] = c0[a];
  if constexpr (D == 3)
    sm[0] = ghost_need3(g, cls, L0, sc[0]);
  else
    sm[0] = ghost_stencil_need<D>(g, cls, L0, sc[0][0], sc[0][1]);
  int sp = 1;
  while (sp > 0) {
    const int t = sp - 1;
    if (sm[t] == 0u) {
      --sp;
      continue;
    }
    const int k = __ffs(sm[t]) - 1;
    sm[t] &= sm[t] - 1u;
    const int L = sl[t];
    int ac[3] = {sc[t][0] + k % 3 - 1, D >= 2 ? sc[t][1] + (k / 3) % 3 - 1 : 0, D == 3 ? sc[t][2] + k / 9 - 1 : 0};
    mr_nbr_mesh_d<D>(g, L, ac);  // inside: only such cells enter the mask
    const uint32_t ga = g.base[L] + mr_encode_d<D>(g, L, ac);
    const uint32_t o2 = mr_atomic_or_byte(cls, ga, MR_C_GHOST);
    if (o2 & MR_C_GHOST) continue;
    mr_touch(act, ga);
    if (L - 1 < g.Jmin || sp >= MR_MAXL) continue;
    for (int a = 0; a < 3; ++a) sc[sp][a] = a < D ? ac[a] >> 1 : 0;
    if (!mr_claim_stencil(cls, act, g.base[L - 1] + mr_encode_d<D>(g, L - 1, sc[sp]))) continue;
    sl[sp] = L - 1;
    if constexpr (D == 3)
      sm[sp] = ghost_need3(g, cls, L - 1, sc[sp]);
    else
      sm[sp] = ghost_stencil_need<D>(g, cls, L - 1, sc[sp][0], sc[sp][1]);
    ++sp;
  }
}

// A block per touched chunk at a time, grid-stride over the chunks of all
// instances (a chunk nothing touched holds no leaf).
template <int D>
__global__ void __launch_bounds__(256) k_mark_ghosts(const InstDev* __restrict__ IB,
                                                     const int* __restrict__ chunk_pre, int n, int nchunks) {
  __shared__ InstDev si;
  __shared__ uint16_t queue[MR_DENSE_ALIGN];  // the chunk's leaves (offsets in the chunk)
  __shared__ int32_t qc[D == 3 ? 3 : 1][D == 3 ? MR_DENSE_ALIGN : 1];  // 3D: their coordinates, decoded once
  __shared__ int qn;
  int have = -1;
  mr_grid_dep();
  for (int t = blockIdx.x; t < nchunks; t += gridDim.x) {
    int chunk;
    const int ib = mr_group_chunk_of(chunk_pre, n, t, chunk);
    // one read for the block (other blocks may touch the byte meanwhile)
    if (!__syncthreads_or(threadIdx.x == 0 && IB[ib].act[chunk])) continue;
    mr_inst_use(si, have, IB, ib);
    const Geo& g = si.g;
    uint8_t* cls = si.cls;
    const bool block = D == 2 && g.diag;
    const uint32_t c0 = (uint32_t)chunk * MR_DENSE_ALIGN;
    const int l = mr_level_of(g, c0);
    const uint32_t cb = c0 - g.base[l];
    if (threadIdx.x == 0) qn = 0;
    __syncthreads();
    // Leaves are a few per cent of the dense cells: gather them first, so that
    // the marking below runs on full warps instead of one lane in 32.  The
    // marks are a union (atomic ORs; only the thread that sets a ghost walks
    // its parent stencil), so the result does not depend on the order.
    {
      const int lane = threadIdx.x & 31;
#pragma unroll
      for (int k = 0; k < (int)(MR_DENSE_ALIGN / 256u); ++k) {
        const uint32_t off = (uint32_t)k * 256u + threadIdx.x;
        const bool leaf = cb + off < g.ncode[l] && (cls[c0 + off] & 3u) == MR_C_LEAF;
        const uint32_t bal = __ballot_sync(0xffffffffu, leaf);
        int at = 0;
        if (lane == 0 && bal) at = atomicAdd(&qn, __popc(bal));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (leaf) {
          const int q = at + __popc(bal & ((1u << lane) - 1u));
          queue[q] = (uint16_t)off;
          if constexpr (D == 3) {
            int c[3];
            mr_decode_d<3>(g, l, cb + off, c);
            qc[0][q] = c[0];
            qc[1][q] = c[1];
            qc[2][q] = c[2];
          }
        }
      }
    }
    __syncthreads();
    const int nq = qn;
    if constexpr (D == 3) {
      // (leaf, window cell) pairs over the whole block: the 12 axis window
      // cells of a leaf are independent, and most are in the tree already
      for (int it = threadIdx.x; it < nq * 12; it += blockDim.x) {
        const int w = it % 12, k = w & 3;
        const int q = it / 12;
        int nb[3] = {qc[0][q], qc[1][q], qc[2][q]};
        nb[w >> 2] += k < 2 ? k - 2 : k - 1;  // -2, -1, +1, +2 along axis w / 4
        if (!mr_nbr_mesh_d<3>(g, l, nb)) continue;
        const uint32_t gw = g.base[l] + mr_encode_d<3>(g, l, nb);
        if (cls[gw] & (3u | MR_C_GHOST)) continue;  // in the tree or marked
        const uint32_t old = mr_atomic_or_byte(cls, gw, MR_C_GHOST);
        if (old & MR_C_GHOST) continue;
        mr_touch(si.act, gw);
        if (l - 1 < g.Jmin) continue;
        const int pc[3] = {nb[0] >> 1, nb[1] >> 1, nb[2] >> 1};
        ghost_cascade<3>(g, cls, si.act, l - 1, pc);
      }
    } else {
    for (int qi = threadIdx.x; qi < nq; qi += blockDim.x) {
      const uint32_t c = cb + queue[qi];
      int x, y;
      mr_decode(g, l, c, x, y);
      uint32_t need = 0;
      const uint8_t* cl = cls + g.base[l];
      if constexpr (D == 2) {
        MortonBox<2> bx;
        bx.init(g, l, x, y);
        if (block) {
#pragma unroll
          for (int w = 0; w < 25; ++w) {
            if (w == 12) continue;  // the leaf itself
            if (bx.in(w % 5, w / 5) && !(cl[bx.code(w % 5, w / 5)] & (3u | MR_C_GHOST))) need |= 1u << w;
          }
        } else {
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            const int axis = w >> 2, k = w & 3;
            const int off = k < 2 ? k - 2 : k - 1;
            const int a = axis == 0 ? 2 + off : 2, b = axis == 1 ? 2 + off : 2;
            if (bx.in(a, b) && !(cl[bx.code(a, b)] & (3u | MR_C_GHOST))) need |= 1u << w;
          }
        }
      } else {
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          int nx, ny;
          ghost_window_cell(false, w, x, y, nx, ny);
          if (!mr_nbr_mesh(g, l, nx, ny)) continue;
          if (!(cl[mr_encode(g, l, nx, ny)] & (3u | MR_C_GHOST))) need |= 1u << w;
        }
      }
      while (need) {
        const int w = __ffs(need) - 1;
        need &= need - 1u;
        int nx, ny;
        ghost_window_cell(block, w, x, y, nx, ny);
        mr_nbr_mesh(g, l, nx, ny);  // inside: only such cells enter the mask
        const uint32_t gw = g.base[l] + mr_encode(g, l, nx, ny);
        const uint32_t old = mr_atomic_or_byte(cls, gw, MR_C_GHOST);
        if (old & MR_C_GHOST) continue;
        mr_touch(si.act, gw);
        if (l - 1 < g.Jmin) continue;
        // cascade: the stencil of the ghost's parent, towards coarser levels
        const int pc[3] = {nx >> 1, ny >> 1, 0};
        ghost_cascade<D>(g, cls, si.act, l - 1, pc);
      }
    }
    }
  }  // the barrier at the top of the next chunk ends this chunk's use of the queue
}

// ---------------------------------------------------------------- compaction
// Stream compaction of the dense classification: class counts per 1024-cell
// chunk (k_count), one scan over the chunks of each instance (k_scan_blocks),
// then every cell written at its position (k_scatter).
__device__ __forceinline__ int cls_of(uint8_t c) {
  const uint32_t k = c & 3u;
  if (k == MR_C_LEAF) return MR_CLS_LEAF;
  if (k == MR_C_INT) return MR_CLS_INT;
  if (c & MR_C_GHOST) return MR_CLS_GHOST;
  return -1;
}

// One warp per 1024-cell chunk, grid-stride over the chunks of all
// instances, no block barrier: lane L reads the class bytes of cells
// 32L .. 32L+31 of the chunk (two 16-byte loads) and counts them four at a
// time with per-byte compares; the three counts are summed over the warp.
__device__ __forceinline__ void cls_count4(uint32_t w, int& nl, int& ni, int& ng) {
  const uint32_t lo = w & 0x03030303u;
  const uint32_t isL = __vcmpeq4(lo, 0x01010101u * MR_C_LEAF);  // 0xFF in every matching byte
  const uint32_t isI = __vcmpeq4(lo, 0x01010101u * MR_C_INT);
  const uint32_t isG = __vcmpne4(w & (0x01010101u * MR_C_GHOST), 0u) & ~isL & ~isI;
  nl += __popc(isL) >> 3;
  ni += __popc(isI) >> 3;
  ng += __popc(isG) >> 3;
}

__global__ void __launch_bounds__(256) k_count(const InstDev* __restrict__ IB, const int* __restrict__ chunk_pre,
                                               int n, int nchunks) {
  mr_grid_dep();
  const int lane = threadIdx.x & 31;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < nchunks; t += nw) {
    int chunk;
    const int b = mr_group_chunk_of(chunk_pre, n, t, chunk);
    if (!IB[b].act[chunk]) {  // nothing classified or marked in it
      if (lane == 0) {
        int* bc = IB[b].bcounts + 3 * chunk;
        bc[0] = bc[1] = bc[2] = 0;
      }
      continue;
    }
    const uint4* src = (const uint4*)(IB[b].cls + (size_t)chunk * MR_DENSE_ALIGN) + 2 * lane;
    const uint4 v0 = src[0], v1 = src[1];
    int nl = 0, ni = 0, ng = 0;
    cls_count4(v0.x, nl, ni, ng);
    cls_count4(v0.y, nl, ni, ng);
    cls_count4(v0.z, nl, ni, ng);
    cls_count4(v0.w, nl, ni, ng);
    cls_count4(v1.x, nl, ni, ng);
    cls_count4(v1.y, nl, ni, ng);
    cls_count4(v1.z, nl, ni, ng);
    cls_count4(v1.w, nl, ni, ng);
    nl = __reduce_add_sync(0xffffffffu, nl);
    ni = __reduce_add_sync(0xffffffffu, ni);
    ng = __reduce_add_sync(0xffffffffu, ng);
    if (lane == 0) {
      int* bc = IB[b].bcounts + 3 * chunk;
      bc[0] = nl;
      bc[1] = ni;
      bc[2] = ng;
    }
  }
}

// Exclusive scan of the chunk counts of one instance (one block per
// instance), the three classes together: each thread takes MR_SCAN_VPT
// consecutive chunks, so that a pass covers 1024 * MR_SCAN_VPT chunks.
#define MR_SCAN_VPT 8
__global__ void __launch_bounds__(1024) k_scan_blocks(const InstDev* __restrict__ IB, int dst) {
  __shared__ int warp_sums[32][3];
  __shared__ int carry[3];
  __shared__ InstDev si;
  int have = -1;
  mr_inst_use(si, have, IB, blockIdx.x);
  mr_grid_dep();  // after the copy of the descriptor, which no step kernel writes
  const Geo& g = si.g;
  int* bc = si.bcounts;
  const int nblocks = (int)(g.base[g.J + 1] / MR_DENSE_ALIGN);
  MeshCounts* cnt = si.mesh[dst].cnt;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x < 3) carry[threadIdx.x] = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nblocks; b0 += 1024 * MR_SCAN_VPT) {
    const int first = b0 + threadIdx.x * MR_SCAN_VPT;
    // the thread's 3 MR_SCAN_VPT counts are consecutive (96 bytes, 16-byte
    // aligned): six 16-byte loads where the chunks are all there
    const bool whole = first + MR_SCAN_VPT <= nblocks;
    int v[MR_SCAN_VPT][3], x[3], tot[3] = {0, 0, 0};
    if (whole) {
      const int4* src = (const int4*)(bc + first * 3);
      int w[3 * MR_SCAN_VPT];
#pragma unroll
      for (int k = 0; k < 3 * MR_SCAN_VPT / 4; ++k) {
        const int4 q = src[k];
        w[4 * k] = q.x;
        w[4 * k + 1] = q.y;
        w[4 * k + 2] = q.z;
        w[4 * k + 3] = q.w;
      }
#pragma unroll
      for (int j = 0; j < MR_SCAN_VPT; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) v[j][c] = w[3 * j + c];
    } else {
#pragma unroll
      for (int j = 0; j < MR_SCAN_VPT; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) v[j][c] = first + j < nblocks ? bc[(first + j) * 3 + c] : 0;
    }
#pragma unroll
    for (int j = 0; j < MR_SCAN_VPT; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) tot[c] += v[j][c];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[c] = tot[c];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x[c], o);
        if (lane >= o) x[c] += y;
      }
      if (lane == 31) warp_sums[wid][c] = x[c];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        int t = warp_sums[lane][c];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, t, o);
          if (lane >= o) t += y;
        }
        warp_sums[lane][c] = t;
      }
    }
    __syncthreads();
    int run[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) run[c] = carry[c] + (wid > 0 ? warp_sums[wid - 1][c] : 0) + x[c] - tot[c];
    int w[3 * MR_SCAN_VPT];
#pragma unroll
    for (int j = 0; j < MR_SCAN_VPT; ++j)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        w[3 * j + c] = run[c];
        run[c] += v[j][c];
      }
    if (whole) {
      int4* dst4 = (int4*)(bc + first * 3);
#pragma unroll
      for (int k = 0; k < 3 * MR_SCAN_VPT / 4; ++k) dst4[k] = make_int4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < MR_SCAN_VPT; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (first + j < nblocks) bc[(first + j) * 3 + c] = w[3 * j + c];
    }
    __syncthreads();  // every thread has read carry
    if (threadIdx.x == 1023)
#pragma unroll
      for (int c = 0; c < 3; ++c) carry[c] = run[c];
    __syncthreads();
  }
  // per-level offsets (every level starts on a block boundary), one thread
  // per class and level so that the loads are issued together; counts are
  // clamped to the capacity so that no later kernel can run past an array,
  // and the overflow itself is reported through err
  if (threadIdx.x < 3 * (MR_MAXL + 1)) {
    const int c = threadIdx.x % 3, l = threadIdx.x / 3;
    const int total = carry[c] < g.cap[c] ? carry[c] : g.cap[c];
    int v;
    if (l < g.Jmin)
      v = 0;
    else if (l <= g.J)
      v = bc[(g.base[l] / MR_DENSE_ALIGN) * 3 + c];
    else
      v = total;
    cnt->off[c][l] = v < g.cap[c] ? v : g.cap[c];
    if (l == 0) {
      cnt->total[c] = total;
      if (carry[c] > g.cap[c]) atomicOr(&cnt->err, MR_DERR_CAPACITY);
    }
  }
}

// One warp per chunk, as k_count, with no block barrier: the warp walks the
// chunk's cells 32 at a time in index order (lane L takes cell 32 it + L),
// the position of each cell in its class array being the chunk's offset
// plus the ballot prefix, so that every write is coalesced and every cell
// gets its place in (level, code) order.  The class bytes, read up front,
// and the flag bytes are then cleared 16 bytes at a time.
__global__ void __launch_bounds__(256) k_scatter(const InstDev* __restrict__ IB, const int* __restrict__ chunk_pre,
                                                 int n, int dst, int nchunks) {
  mr_grid_dep();
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < nchunks; t += nw) {
    int chunk;
    const InstDev& I = IB[mr_group_chunk_of(chunk_pre, n, t, chunk)];
    const Geo& g = I.g;
    const MeshDev& B = I.mesh[dst];
    const uint32_t c0 = (uint32_t)chunk * MR_DENSE_ALIGN;
    const bool touched = I.act[chunk], held = B.mact[chunk];
    if (!touched) {
      if (held) {  // entries of the mesh last written here: clear them
        const int4 none = make_int4(MR_MAP_NONE, MR_MAP_NONE, MR_MAP_NONE, MR_MAP_NONE);
        int4* mp = (int4*)(B.map + c0);
#pragma unroll
        for (int k = 0; k < 8; ++k) mp[32 * k + lane] = none;
        if (lane == 0) B.mact[chunk] = 0;
      }
      continue;
    }
    const uint8_t* cl = I.cls + c0;
    uint8_t v[32];
#pragma unroll
    for (int it = 0; it < 32; ++it) v[it] = cl[32 * it + lane];
    int run0 = I.bcounts[3 * chunk + 0], run1 = I.bcounts[3 * chunk + 1], run2 = I.bcounts[3 * chunk + 2];
    const int l = mr_level_of(g, c0);
    const uint32_t cb = c0 - g.base[l];
    int32_t* map = B.map + c0;
#pragma unroll
    for (int it = 0; it < 32; ++it) {
      const int k = cls_of(v[it]);
      const uint32_t bl = __ballot_sync(0xffffffffu, k == (int)MR_CLS_LEAF);
      const uint32_t bi = __ballot_sync(0xffffffffu, k == (int)MR_CLS_INT);
      const uint32_t bg = __ballot_sync(0xffffffffu, k == (int)MR_CLS_GHOST);
      const int at = k == (int)MR_CLS_LEAF ? run0 + __popc(bl & lt)
                                           : (k == (int)MR_CLS_INT ? run1 + __popc(bi & lt) : run2 + __popc(bg & lt));
      run0 += __popc(bl);
      run1 += __popc(bi);
      run2 += __popc(bg);
      int32_t e = MR_MAP_NONE;
      if (k >= 0 && at < g.cap[k]) {
        B.code[k][at] = cb + 32u * (uint32_t)it + (uint32_t)lane;
        B.lvl[k][at] = (uint8_t)l;
        e = (int32_t)(((uint32_t)k << 30) | (uint32_t)at);
      }
      map[32 * it + lane] = e;
    }
    __syncwarp();  // every lane's class bytes are read before any are cleared
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    uint4* clp = (uint4*)(I.cls + c0) + 2 * lane;
    uint4* flp = (uint4*)(I.flags + c0) + 2 * lane;
    clp[0] = zero;
    clp[1] = zero;
    flp[0] = zero;
    flp[1] = zero;
    if (lane == 0) {
      B.mact[chunk] = 1;
      I.act[chunk] = 0;
      I.acth[chunk] = 0;
    }
  }
}

// ---------------------------------------------------------------- input leaves
template <int D>
__global__ void __launch_bounds__(256) k_leaves_in(Geo g, long long n, const unsigned long long* keys,
                                                   const signed char* levels, int32_t* inidx,
                                                   uint8_t* cls, uint8_t* act, MeshCounts* cnt,
                                                   unsigned long long* vol) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int l = levels[i];
    const unsigned long long key = keys[i];
    if (l < g.Jmin || l > g.J || key >= g.ncode[l]) {
      mr_set_err(cnt, MR_DERR_INPUT);
      continue;
    }
    const uint32_t c = (uint32_t)key;
    const uint32_t old = mr_atomic_or_byte(cls, g.base[l] + c, MR_C_LEAF);
    mr_touch(act, g.base[l] + c);
    if (old & MR_C_LEAF) mr_set_err(cnt, MR_DERR_INPUT);
    inidx[g.base[l] + c] = (int32_t)i;
    atomicAdd(vol, 1ull << (D * (g.J - l)));
    uint32_t a = c;
    for (int la = l - 1; la >= g.Jmin; --la) {
      a >>= D;
      const uint32_t o = mr_atomic_or_byte(cls, g.base[la] + a, MR_C_INT);
      if (o & MR_C_INT) break;
      mr_touch(act, g.base[la] + a);
    }
  }
}

__global__ void __launch_bounds__(256) k_leaves_check(Geo g, const uint8_t* __restrict__ cls,
                                                      MeshCounts* cnt) {
  const uint32_t lo = g.base[g.Jmin], hi = g.base[g.J + 1];
  for (uint32_t gi = lo + blockIdx.x * blockDim.x + threadIdx.x; gi < hi; gi += gridDim.x * blockDim.x)
    if ((cls[gi] & 3u) == 3u) mr_set_err(cnt, MR_DERR_INPUT);
}

}  // namespace

#define MR_DISPATCH_D(KER, GRID, BLOCK, SMEM, ST, ...)           \
  do {                                                           \
    if (D_ == 1)                                                 \
      KER<1><<<GRID, BLOCK, SMEM, ST>>>(__VA_ARGS__);            \
    else if (D_ == 2)                                            \
      KER<2><<<GRID, BLOCK, SMEM, ST>>>(__VA_ARGS__);            \
    else                                                         \
      KER<3><<<GRID, BLOCK, SMEM, ST>>>(__VA_ARGS__);            \
  } while (0)
// step kernels (they call mr_grid_dep before reading what an earlier kernel writes)
#define MR_DISPATCH_D_PDL(KER, GRID, BLOCK, SMEM, ST, ...)                 \
  do {                                                                     \
    if (D_ == 1)                                                           \
      mr_launch_pdl(KER<1>, GRID, BLOCK, SMEM, ST, __VA_ARGS__);           \
    else if (D_ == 2)                                                      \
      mr_launch_pdl(KER<2>, GRID, BLOCK, SMEM, ST, __VA_ARGS__);           \
    else                                                                   \
      mr_launch_pdl(KER<3>, GRID, BLOCK, SMEM, ST, __VA_ARGS__);           \
  } while (0)

void mr_launch_flags_T(const Group& G, int cur, cudaStream_t st) {
  const int D_ = G.d;
  MR_DISPATCH_D_PDL(k_flags_T, mr_tile_grid(G, G.capI, 256, G.bps[MR_PH_FLAGS]), 256, mr_pre_bytes(G), st, G.dev, G.n, cur);
}
void mr_launch_flags_H(const Group& G, int cur, cudaStream_t st) {
  const int D_ = G.d;
  MR_DISPATCH_D_PDL(k_flags_H, mr_tile_grid(G, G.capI, 256, G.bps[MR_PH_FLAGS]), 256, mr_pre_bytes(G), st, G.dev, G.n, cur);
}
void mr_launch_grade(const Group& G, cudaStream_t st) {
  if (G.s > 1) return mr_launch_grade_w(G, st);
  const int D_ = G.d;
  if (G.grade)
    MR_DISPATCH_D_PDL(k_grade, mr_tile_grid(G, (long long)G.chunks * MR_DENSE_ALIGN, 256, G.bps[MR_PH_FLAGS]), 256, mr_pre_bytes(G), st,
                  G.dev, G.n);
}
// dense kernels: grid-stride over the 1024-cell chunks of every instance,
// visiting the touched ones
int mr_chunk_warps_grid(const Group& G) {  // one warp per chunk, 8 warps per block
  return std::max(1, std::min((G.chunks + 7) / 8, G.bps[MR_PH_COMPACT] * G.nsm));
}
void mr_launch_classify(const Group& G, cudaStream_t st) {
  const int D_ = G.d;
  MR_DISPATCH_D_PDL(k_classify, mr_chunk_warps_grid(G), 256, 0, st, G.dev, G.chunk_pre, G.n, G.chunks);
}
void mr_launch_full_mesh(const Geo& g, uint8_t* cls, uint8_t* act, cudaStream_t st, int) {
  k_full_mesh<<<(int)(g.base[g.J + 1] / MR_DENSE_ALIGN), 256, 0, st>>>(g, cls, act);
}
int mr_chunk_blocks_grid(const Group& G) {  // one block per chunk: an untouched one ends at once
  return std::max(1, G.chunks);
}
void mr_launch_mark_ghosts(const Group& G, cudaStream_t st) {
  if (G.s > 1) return mr_launch_mark_ghosts_w(G, st);
  const int D_ = G.d;
  MR_DISPATCH_D_PDL(k_mark_ghosts, mr_chunk_blocks_grid(G), 256, 0, st, G.dev, G.chunk_pre, G.n, G.chunks);
}
void mr_launch_compact(const Group& G, int dst, cudaStream_t st) {
  const int grid = mr_chunk_warps_grid(G);
  mr_launch_pdl(k_count, grid, 256, 0, st, G.dev, G.chunk_pre, G.n, G.chunks);
  mr_launch_pdl(k_scan_blocks, G.n, 1024, 0, st, G.dev, dst);
  mr_launch_pdl(k_scatter, grid, 256, 0, st, G.dev, G.chunk_pre, G.n, dst, G.chunks);
}
void mr_launch_leaves_in(const Geo& g, long long n, const unsigned long long* keys,
                         const signed char* levels, int32_t* inidx, uint8_t* cls, uint8_t* act, MeshCounts* cnt,
                         unsigned long long* vol, cudaStream_t st, int grid) {
  const int D_ = g.d;
  MR_DISPATCH_D(k_leaves_in, grid, 256, 0, st, g, n, keys, levels, inidx, cls, act, cnt, vol);
}
void mr_launch_leaves_check(const Geo& g, uint8_t* cls, MeshCounts* cnt, cudaStream_t st, int grid) {
  k_leaves_check<<<grid, 256, 0, st>>>(g, cls, cnt);
}

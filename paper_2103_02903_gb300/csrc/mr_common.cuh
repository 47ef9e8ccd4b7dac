// Device helpers shared by the kernels: value lookup through the dense index
// map, byte atomics, grid-stride ranges and the canonical prediction
// operator of Sec. 4.1 (s = 1).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mr_internal.cuh"

#define MR_C1 (-0.125)  // Table 1, s = 1

// ------------------------------------------------------------------ forms
// S: storage type of the populations, C: arithmetic of transport and
// collision, offs: stored value = population - g.off[p].
template <int F>
struct FormT;
template <>
struct FormT<MR_FORM_F64> {
  using S = double;
  using C = double;
  static constexpr bool offs = false;
};
template <>
struct FormT<MR_FORM_F32> {
  using S = float;
  using C = float;
  static constexpr bool offs = false;
};
template <>
struct FormT<MR_FORM_F32_F16> {
  using S = __half;
  using C = float;
  static constexpr bool offs = true;
};
template <>
struct FormT<MR_FORM_F32_BF16> {
  using S = __nv_bfloat16;
  using C = float;
  static constexpr bool offs = true;
};

__device__ __forceinline__ double mr_cvt_d(double v) { return v; }
__device__ __forceinline__ double mr_cvt_d(float v) { return (double)v; }
__device__ __forceinline__ double mr_cvt_d(__half v) { return (double)__half2float(v); }
__device__ __forceinline__ double mr_cvt_d(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <class S>
__device__ __forceinline__ S mr_from_d(double v);
template <>
__device__ __forceinline__ double mr_from_d<double>(double v) { return v; }
template <>
__device__ __forceinline__ float mr_from_d<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __half mr_from_d<__half>(double v) { return __double2half(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 mr_from_d<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

template <class S>
__device__ __forceinline__ S mr_from_f(float v);
template <>
__device__ __forceinline__ double mr_from_f<double>(float v) { return (double)v; }
template <>
__device__ __forceinline__ float mr_from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half mr_from_f<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 mr_from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// A constant of the geometry in the arithmetic type C: the FP64 value, or
// its FP32 copy (MR_K(C, g, s[0]) and the like).
template <class C>
__device__ __forceinline__ C mr_k(double d, float) {
  return C(d);
}
template <>
__device__ __forceinline__ float mr_k<float>(double, float f) { return f; }
#define MR_K(C, g, field) mr_k<C>((g).field, (g).f32.field)

// The flattened-weight table in the arithmetic type C.
template <class C>
__device__ __forceinline__ const C* mr_wtab(const InstDev& si);
template <>
__device__ __forceinline__ const double* mr_wtab<double>(const InstDev& si) { return si.W; }
template <>
__device__ __forceinline__ const float* mr_wtab<float>(const InstDev& si) { return si.Wf; }

// Prologue of a step kernel launched with mr_launch_pdl: wait for the
// preceding grid (a no-op when there is none in flight), then allow the
// next one to be scheduled.
__device__ __forceinline__ void mr_grid_dep() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Storage offsets of the populations (Geo::off) in the arithmetic C.
template <class C>
__device__ __forceinline__ const C* mr_offv(const Geo& g) {
  return g.off;
}
template <>
__device__ __forceinline__ const float* mr_offv<float>(const Geo& g) {
  return g.f32.off;
}

// A cell's population array: element p is at p[p * stride].
template <class S = double>
struct ValPtr {
  const S* p;
  int stride;
};

template <class S = double>
__device__ __forceinline__ ValPtr<S> mr_resolve(const Geo& g, const MeshDev& M, const void* LF, int32_t e) {
  uint32_t cls = ((uint32_t)e) >> 30;
  uint32_t idx = (uint32_t)e & 0x3FFFFFFFu;
  ValPtr<S> r;
  if (cls == MR_CLS_LEAF) {
    r.p = (const S*)LF + idx;
    r.stride = g.cap[0];
  } else if (cls == MR_CLS_INT) {
    r.p = (const S*)M.IF + idx;
    r.stride = g.cap[1];
  } else {
    r.p = (const S*)M.GF + idx;
    r.stride = g.cap[2];
  }
  return r;
}

// stored value of population p as double (no offset added)
template <class S>
__device__ __forceinline__ double mr_ld(const ValPtr<S>& v, int p) {
  return mr_cvt_d(__ldg(v.p + (size_t)p * v.stride));
}

__device__ __forceinline__ uint32_t mr_atomic_or_byte(uint8_t* base, uint32_t idx, uint32_t bits) {
  uint32_t* w = (uint32_t*)(base + (idx & ~3u));
  uint32_t sh = (idx & 3u) * 8u;
  uint32_t old = atomicOr(w, bits << sh);
  return (old >> sh) & 0xFFu;
}

__device__ __forceinline__ void mr_set_err(MeshCounts* c, int bits) { atomicOr(&c->err, bits); }

// The cell of dense index gi was flagged, classified or marked: the dense
// passes of this step visit its 1024-cell chunk (every writer stores 1).
__device__ __forceinline__ void mr_touch(uint8_t* act, uint32_t gi) { act[gi / MR_DENSE_ALIGN] = 1; }

// Ghost marking: the stencil around the cell of dense index gi (the parent of
// a new ghost) is walked by the one thread that claims it first, so that
// sibling ghosts and overlapping cascades walk each stencil once.
__device__ __forceinline__ bool mr_claim_stencil(uint8_t* cls, uint8_t* act, uint32_t gi) {
  if (cls[gi] & MR_C_STEN) return false;  // a plain load first
  if (mr_atomic_or_byte(cls, gi, MR_C_STEN) & MR_C_STEN) return false;
  mr_touch(act, gi);
  return true;
}

// level of a dense index (levels J_min..J)
__device__ __forceinline__ int mr_level_of(const Geo& g, uint32_t gi) {
  int l = g.Jmin;
  while (l < g.J && gi >= g.base[l + 1]) ++l;
  return l;
}

// Dense kernels run one block of 256 threads per 1024-cell chunk of the dense
// index space; CHUNK is the block's chunk.  Every level starts on a chunk
// boundary, so a block finds its level once; the body sees the level L, the
// code C and the dense index GI of each valid cell of the chunk.
#define MR_DENSE_CHUNK_BEGIN(g, CHUNK, L, C, GI)                               \
  {                                                                           \
    const uint32_t mr_chunk_ = (CHUNK);                                       \
    const int L = mr_level_of(g, mr_chunk_ * MR_DENSE_ALIGN);                 \
    const uint32_t mr_cb_ = mr_chunk_ * MR_DENSE_ALIGN - (g).base[L];         \
    for (int mr_k_ = 0; mr_k_ < (int)(MR_DENSE_ALIGN / 256u); ++mr_k_) {      \
      const uint32_t C = mr_cb_ + (uint32_t)mr_k_ * 256u + threadIdx.x;       \
      if (C >= (g).ncode[L]) break;                                           \
      const uint32_t GI = (g).base[L] + C;
#define MR_DENSE_CHUNK_END \
  }                        \
  }

// ------------------------------------------------------------------ boxes
// Morton codes of a box of cells around (x, y) on level l (d = 2).  The code
// of cell (X, Y) is (root << 2l) | spread(X mod 2^l) | spread(Y mod 2^l) << 1
// with root = (X >> l) + roots_x (Y >> l): a sum of a part of X and a part
// of Y, so the (2R+1)^2 codes of the box come from 2R+1 column parts and
// 2R+1 row parts (a few integer operations per cell instead of a full
// interleave).  Columns and rows are x + o - R, o = 0..2R, wrapped on a
// periodic axis; ix / iy are false for one outside a non-periodic domain.
// With `half` the codes are those of the parents (X >> 1, Y >> 1), on level
// l - 1, of the (wrapped) level-l cells.
template <int R>
struct MortonBox {
  static constexpr int W = 2 * R + 1;
  uint32_t px[W], rx[W], py[W], ry[W];
  bool ix[W], iy[W];
  int sh;
  __device__ __forceinline__ void init(const Geo& g, int l, int x, int y, bool half = false) {
    const int Nx = g.n[l][0], Ny = g.n[l][1];
    const int lc = half ? l - 1 : l;
    const uint32_t mask = (1u << lc) - 1u;
    sh = 2 * lc;
#pragma unroll
    for (int o = 0; o < W; ++o) {
      int X = x + o - R, Y = y + o - R;
      ix[o] = X >= 0 && X < Nx;
      if (!ix[o] && g.periodic[0]) {
        X = mr_wrap(X, Nx);
        ix[o] = true;
      }
      iy[o] = Y >= 0 && Y < Ny;
      if (!iy[o] && g.periodic[1]) {
        Y = mr_wrap(Y, Ny);
        iy[o] = true;
      }
      if (half) {
        X >>= 1;
        Y >>= 1;
      }
      px[o] = mr_spread2((uint32_t)X & mask);
      rx[o] = (uint32_t)X >> lc;
      py[o] = mr_spread2((uint32_t)Y & mask) << 1;
      ry[o] = (uint32_t)g.roots[0] * ((uint32_t)Y >> lc);
    }
  }
  __device__ __forceinline__ bool in(int a, int b) const { return ix[a] && iy[b]; }
  __device__ __forceinline__ uint32_t code(int a, int b) const { return ((rx[a] + ry[b]) << sh) | px[a] | py[b]; }
};

// d = 3 form of MortonBox: the code of (X, Y, Z) is the sum of an X part, a
// Y part and a Z part (root X >> l + roots_x (Y >> l + roots_y (Z >> l))
// shifted by 3l, or-ed with the three 3-way interleaves), so a box needs
// 3 (2R+1) interleaves.  Same wrap / outside / `half` rules as MortonBox.
template <int R>
struct MortonBox3 {
  static constexpr int W = 2 * R + 1;
  uint32_t p[3][W], r[3][W];
  bool in[3][W];
  int sh;
  __device__ __forceinline__ void init(const Geo& g, int l, const int* c, bool half = false) {
    const int lc = half ? l - 1 : l;
    const uint32_t mask = (1u << lc) - 1u;
    const uint32_t rs[3] = {1u, (uint32_t)g.roots[0], (uint32_t)g.roots[0] * (uint32_t)g.roots[1]};
    sh = 3 * lc;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int o = 0; o < W; ++o) {
        int X = c[a] + o - R;
        const int n = g.n[l][a];
        in[a][o] = X >= 0 && X < n;
        if (!in[a][o] && g.periodic[a]) {
          X = mr_wrap(X, n);
          in[a][o] = true;
        }
        if (half) X >>= 1;
        p[a][o] = mr_spread3((uint32_t)X & mask) << a;
        r[a][o] = rs[a] * ((uint32_t)X >> lc);
      }
  }
  __device__ __forceinline__ bool inside(int i, int j, int k) const { return in[0][i] && in[1][j] && in[2][k]; }
  __device__ __forceinline__ uint32_t code(int i, int j, int k) const {
    return ((r[0][i] + r[1][j] + r[2][k]) << sh) | p[0][i] | p[1][j] | p[2][k];
  }
};

// ------------------------------------------------------------------ groups
// A step kernel runs one phase for every instance of a group.  The phase's
// work in instance b is count(b) passes of the block ("tiles"); the tiles of
// all instances are numbered in instance order and the blocks stride over
// them, so the work of uneven instances is spread over the whole grid.
// pre (shared, n + 1 ints) receives the first tile of every instance; the
// return value is the number of tiles.  Block-wide: every thread calls it.
template <class CountF>
__device__ __forceinline__ int mr_group_prefix(int* pre, int n, CountF count) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  if (n == 1) {
    if (tid == 0) {
      pre[0] = 0;
      pre[1] = count(0);
    }
    __syncthreads();
    return pre[1];
  }
  for (int b = tid; b < n; b += nt) pre[b + 1] = count(b);
  __syncthreads();
  if (tid < 32) {
    // each lane scans a run of entries, then the runs are offset by a warp scan
    const int per = (n + 31) / 32, lo = 1 + tid * per, hi = min(lo + per, n + 1);
    int s = 0;
    for (int b = lo; b < hi; ++b) s += pre[b];
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (tid >= o) x += y;
    }
    int run = x - s;
    for (int b = lo; b < hi; ++b) {
      run += pre[b];
      pre[b] = run;
    }
    if (tid == 0) pre[0] = 0;
  }
  __syncthreads();
  return pre[n];
}

// instance of tile t: the largest b with pre[b] <= t
__device__ __forceinline__ int mr_group_find(const int* pre, int n, int t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// The block's shared copy of the descriptor of instance b (b block-uniform);
// `have` is the instance currently held (-1 before the first).
__device__ __forceinline__ void mr_inst_use(InstDev& si, int& have, const InstDev* __restrict__ IB, int b) {
  if (have == b) return;
  __syncthreads();
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int4* s = reinterpret_cast<const int4*>(IB + b);
  int4* d = reinterpret_cast<int4*>(&si);
  for (int k = tid; k < (int)(sizeof(InstDev) / sizeof(int4)); k += nt) d[k] = __ldg(s + k);
  __syncthreads();
  have = b;
}

// Group of one: start copying the only descriptor before the tile prefix,
// whose barrier then publishes it (saves a round trip per kernel).
__device__ __forceinline__ void mr_inst_prefetch(InstDev& si, int& have, const InstDev* __restrict__ IB, int n) {
  if (n != 1) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int4* s = reinterpret_cast<const int4*>(IB);
  int4* d = reinterpret_cast<int4*>(&si);
  for (int k = tid; k < (int)(sizeof(InstDev) / sizeof(int4)); k += nt) d[k] = __ldg(s + k);
  have = 0;
}

// Dense kernels: instance and chunk of this block, from the group's chunk
// prefix (one block per dense chunk of every instance).
__device__ __forceinline__ int mr_group_chunk_of(const int* __restrict__ chunk_pre, int n, int t, int& chunk) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(chunk_pre + mid) <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  chunk = t - __ldg(chunk_pre + lo);
  return lo;
}
__device__ __forceinline__ int mr_group_chunk(const int* __restrict__ chunk_pre, int n, int& chunk) {
  int lo = 0, hi = n - 1;
  const int t = (int)blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(chunk_pre + mid) <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  chunk = t - __ldg(chunk_pre + lo);
  return lo;
}

// All 2^D children of one stencil, each operation rounded as written (FP64,
// no contraction; the oracle's order):
// the products with the signs +-1 are exact, so they become the signs of the
// additions (x + (-y) and x - y round alike), and the partial sums that two
// children share are formed once.  out[ci], ci = x bit | y bit << 1.
template <int D>
__device__ __forceinline__ void mr_predict_children_canonical(const double* v, int cross_sign, double* out) {
  if constexpr (D == 1) {
    const double q = __dmul_rn(MR_C1, __dsub_rn(v[2], v[0]));
    out[0] = __dadd_rn(v[1], q);
    out[1] = __dsub_rn(v[1], q);
  } else if constexpr (D == 2) {
    const double qx = __dmul_rn(MR_C1, __dsub_rn(v[5], v[3]));
    const double qy = __dmul_rn(MR_C1, __dsub_rn(v[7], v[1]));
    const double q2 = __dmul_rn(MR_C1 * MR_C1, __dadd_rn(__dsub_rn(__dsub_rn(v[8], v[6]), v[2]), v[0]));
    const double a = __dadd_rn(v[4], qx), b = __dsub_rn(v[4], qx);
    const double t0 = __dadd_rn(a, qy), t1 = __dadd_rn(b, qy), t2 = __dsub_rn(a, qy), t3 = __dsub_rn(b, qy);
    if (cross_sign > 0) {
      out[0] = __dadd_rn(t0, q2);
      out[1] = __dsub_rn(t1, q2);
      out[2] = __dsub_rn(t2, q2);
      out[3] = __dadd_rn(t3, q2);
    } else {
      out[0] = __dsub_rn(t0, q2);
      out[1] = __dadd_rn(t1, q2);
      out[2] = __dadd_rn(t2, q2);
      out[3] = __dsub_rn(t3, q2);
    }
  } else {
    // d = 3: the tensor product of the one-dimensional operator, terms added
    // in the order x, y, z, xy, xz, yz, xyz (pairs carrying cross_sign)
#define MR_V3(a, b, c) v[(((c) + 1) * 3 + ((b) + 1)) * 3 + ((a) + 1)]
    const double qx = __dmul_rn(MR_C1, __dsub_rn(MR_V3(1, 0, 0), MR_V3(-1, 0, 0)));
    const double qy = __dmul_rn(MR_C1, __dsub_rn(MR_V3(0, 1, 0), MR_V3(0, -1, 0)));
    const double qz = __dmul_rn(MR_C1, __dsub_rn(MR_V3(0, 0, 1), MR_V3(0, 0, -1)));
    const double qxy = __dmul_rn(MR_C1 * MR_C1, __dadd_rn(__dsub_rn(__dsub_rn(MR_V3(1, 1, 0), MR_V3(-1, 1, 0)),
                                                                     MR_V3(1, -1, 0)), MR_V3(-1, -1, 0)));
    const double qxz = __dmul_rn(MR_C1 * MR_C1, __dadd_rn(__dsub_rn(__dsub_rn(MR_V3(1, 0, 1), MR_V3(-1, 0, 1)),
                                                                     MR_V3(1, 0, -1)), MR_V3(-1, 0, -1)));
    const double qyz = __dmul_rn(MR_C1 * MR_C1, __dadd_rn(__dsub_rn(__dsub_rn(MR_V3(0, 1, 1), MR_V3(0, -1, 1)),
                                                                     MR_V3(0, 1, -1)), MR_V3(0, -1, -1)));
    double w = __dsub_rn(MR_V3(1, 1, 1), MR_V3(-1, 1, 1));
    w = __dsub_rn(w, MR_V3(1, -1, 1));
    w = __dsub_rn(w, MR_V3(1, 1, -1));
    w = __dadd_rn(w, MR_V3(-1, -1, 1));
    w = __dadd_rn(w, MR_V3(-1, 1, -1));
    w = __dadd_rn(w, MR_V3(1, -1, -1));
    w = __dsub_rn(w, MR_V3(-1, -1, -1));
    const double q3 = __dmul_rn(MR_C1 * MR_C1 * MR_C1, w);
    const double t0 = MR_V3(0, 0, 0);
#undef MR_V3
#pragma unroll
    for (int ci = 0; ci < 8; ++ci) {
      const int sx = (ci & 1) ? -1 : 1, sy = (ci & 2) ? -1 : 1, sz = (ci & 4) ? -1 : 1;
      // t + s q with s = +-1 is t + q or t - q, bit for bit
      auto add = [](double t, int s, double q) { return s > 0 ? __dadd_rn(t, q) : __dsub_rn(t, q); };
      double t = add(t0, sx, qx);
      t = add(t, sy, qy);
      t = add(t, sz, qz);
      t = add(t, cross_sign * sx * sy, qxy);
      t = add(t, cross_sign * sx * sz, qxz);
      t = add(t, cross_sign * sy * sz, qyz);
      out[ci] = add(t, sx * sy * sz, q3);
    }
  }
}

// Same operator with contraction allowed (used off the decision path).
template <int D>
__device__ __forceinline__ double mr_predict_fast(const double* v, int ci, double cross_sign) {
  const double sx = (ci & 1) ? -1.0 : 1.0;
  if (D == 1) {
    return v[1] + sx * (MR_C1 * (v[2] - v[0]));
  } else {
    const double sy = (ci & 2) ? -1.0 : 1.0;
    double qx = MR_C1 * (v[5] - v[3]);
    double qy = MR_C1 * (v[7] - v[1]);
    double q2 = (MR_C1 * MR_C1) * (((v[8] - v[6]) - v[2]) + v[0]);
    return v[4] + sx * qx + sy * qy + (cross_sign * sx * sy) * q2;
  }
}

// Gather the 3^D stencil entries around (x, y) at level l (constant
// extension outside a non-periodic domain, wrap on periodic axes).
template <int D>
__device__ __forceinline__ bool mr_stencil_entries(const Geo& g, const MeshDev& M, int l, int x, int y,
                                                   int32_t* ent) {
  bool ok = true;
  const int ny3 = D == 2 ? 3 : 1;
  for (int b = 0; b < ny3; ++b)
    for (int a = 0; a < 3; ++a) {
      int sx = x + a - 1, sy = D == 2 ? y + b - 1 : 0;
      mr_nbr_stencil(g, l, sx, sy);
      int32_t e = M.map[g.base[l] + mr_encode(g, l, sx, sy)];
      ent[b * 3 + a] = e;
      ok = ok && (e != MR_MAP_NONE);
    }
  return ok;
}

// Coordinate-array forms (any D): entry e (x fastest) of the 3^D stencil of
// the cell c on level l, and all of them.
template <int D>
__device__ __forceinline__ int32_t mr_stencil_entry_d(const Geo& g, const MeshDev& M, int l, const int* c, int e) {
  int s[3] = {c[0] + (e % 3) - 1, D >= 2 ? c[1] + (e / 3) % 3 - 1 : 0, D == 3 ? c[2] + e / 9 - 1 : 0};
  mr_nbr_stencil_d<D>(g, l, s);
  return M.map[g.base[l] + mr_encode_d<D>(g, l, s)];
}
template <int D>
__device__ __forceinline__ bool mr_stencil_entries_d(const Geo& g, const MeshDev& M, int l, const int* c,
                                                     int32_t* ent) {
  if constexpr (D <= 2) {
    return mr_stencil_entries<D>(g, M, l, c[0], D == 2 ? c[1] : 0, ent);
  } else {
    bool ok = true;
#pragma unroll 1
    for (int e = 0; e < 27; ++e) {
      ent[e] = mr_stencil_entry_d<3>(g, M, l, c, e);
      ok = ok && (ent[e] != MR_MAP_NONE);
    }
    return ok;
  }
}

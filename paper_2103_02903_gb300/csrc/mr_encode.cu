// Multiresolution encode of the stored field (Sec. 4.1-4.2): bottom-up
// projection of the leaves into the internal cells of R(Lambda)
// (Def. Projection) and the details of every cell of R(Lambda) above J_min
// reduced to one max-norm per sibling group and over all populations
// (Def. Details and the group norm of Sec. 4.4).
//
// Both kernels evaluate their arithmetic in FP64, in a fixed order with
// __dadd_rn/__dmul_rn (never contracted into FMA), so that the details, and
// hence every keep / refine decision, carry the same bits as the CPU oracle
// on the same stored values, whatever the storage type of the form.  Both
// act on stored values directly: the projection and the details are linear
// and exact on constants, so the offset of the 16-bit forms cancels.
#include "mr_common.cuh"

namespace {

// Thread layout of the encode kernels: a block is 32 cells (threadIdx.x) by
// up to 8 populations (threadIdx.y), so a warp handles one population of 32
// consecutive cells: its loads are independent of its stores and coalesce
// where the cells' children are consecutive.
template <int Q>
struct PopRows {
  static constexpr int value = Q < 8 ? Q : 8;
};

template <int D, int Q, int F>
__global__ void __launch_bounds__(256) k_project(const InstDev* __restrict__ IB, int n, int cur, int k) {
  using S = typename FormT<F>::S;
  constexpr int PY = PopRows<Q>::value;
  extern __shared__ int pre[];
  __shared__ InstDev si;
  int have = -1;
  mr_inst_prefetch(si, have, IB, n);
  mr_grid_dep();  // after the copy of the descriptor, which no step kernel writes
  const int tiles = mr_group_prefix(pre, n, [&](int b) {
    const InstDev& I = IB[b];
    const int L = I.g.J - k;
    if (L < I.g.Jmin) return 0;
    const MeshCounts* c = I.mesh[cur].cnt;
    return (c->off[MR_CLS_INT][L + 1] - c->off[MR_CLS_INT][L] + 31) / 32;
  });
  const double scale = D == 1 ? 0.5 : D == 2 ? 0.25 : 0.125;  // 2^-d
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int b = mr_group_find(pre, n, t);
    mr_inst_use(si, have, IB, b);
    const Geo& g = si.g;
    const MeshDev& A = si.mesh[cur];
    const int level = g.J - k;
    const int i = A.cnt->off[MR_CLS_INT][level] + (t - pre[b]) * 32 + threadIdx.x;
    if (i >= A.cnt->off[MR_CLS_INT][level + 1]) continue;
    const void* LF = si.fstate;
    S* IF = (S*)A.IF;
    const uint32_t code = A.code[MR_CLS_INT][i];
    ValPtr<S> ch[1 << D];
    bool ok = true;
#pragma unroll
    for (int ci = 0; ci < (1 << D); ++ci) {
      int32_t e = A.map[g.base[level + 1] + ((code << D) | (uint32_t)ci)];
      ok = ok && e != MR_MAP_NONE && (((uint32_t)e) >> 30) <= MR_CLS_INT;
      ch[ci] = mr_resolve<S>(g, A, LF, e);
    }
    if (!ok) {
      if (threadIdx.y == 0) mr_set_err(A.cnt, MR_DERR_INTERNAL);
      continue;
    }
#pragma unroll
    for (int p = threadIdx.y; p < Q; p += PY) {
      double acc = 0.0;
#pragma unroll
      for (int ci = 0; ci < (1 << D); ++ci) acc = __dadd_rn(acc, mr_ld(ch[ci], p));
      IF[(size_t)p * g.cap[1] + i] = mr_from_d<S>(__dmul_rn(acc, scale));
    }
  }
}

// Details of one population of a sibling group in FP16 storage, on the
// integer pipe.  A finite half is an integer multiple of 2^-24 below 2^16 in
// magnitude, so every operation of the canonical FP64 prediction (sums of at
// most four values, products with 1/8 and 1/64) and the difference with
// the child are exact in FP64: the details are these exact values, which
// 64-bit integers in units of 2^-30 reproduce (|value| < 2^50).  The largest
// |detail| is folded into imax.  Returns false (nothing done) when a value
// is not finite: the FP64 path then handles that population.
__device__ __forceinline__ long long half_units30(__half h) {
  const unsigned int b = __half_as_ushort(h);
  const int e = (int)((b >> 10) & 31u), m = (int)(b & 1023u);
  const long long a = e ? (long long)(1024 | m) << (e - 1) : (long long)m;  // |h| 2^24
  return (b & 0x8000u) ? -64 * a : 64 * a;
}

template <int D>
__device__ __forceinline__ bool half_details(const ValPtr<__half>* sv, const ValPtr<__half>* cv, int p,
                                             double cross_sign, long long& imax) {
  if constexpr (D == 3) return false;  // d = 3 keeps the FP64 path
  constexpr int NS = D == 2 ? 9 : 3;
  __half hv[NS], hc[1 << D];
  unsigned int nonfinite = 0;
#pragma unroll
  for (int kk = 0; kk < NS; ++kk) {
    hv[kk] = __ldg(sv[kk].p + (size_t)p * sv[kk].stride);
    nonfinite |= ((__half_as_ushort(hv[kk]) & 0x7c00u) == 0x7c00u);
  }
#pragma unroll
  for (int ci = 0; ci < (1 << D); ++ci) {
    hc[ci] = __ldg(cv[ci].p + (size_t)p * cv[ci].stride);
    nonfinite |= ((__half_as_ushort(hc[ci]) & 0x7c00u) == 0x7c00u);
  }
  if (nonfinite) return false;
  long long w[NS], pr[1 << D];
#pragma unroll
  for (int kk = 0; kk < NS; ++kk) w[kk] = half_units30(hv[kk]);
  // the canonical prediction, exactly: c1 = -1/8, c1^2 = 1/64 (the operands
  // are multiples of 64, so the shifts divide exactly)
  if constexpr (D == 1) {
    const long long q = -((w[2] - w[0]) >> 3);
    pr[0] = w[1] + q;
    pr[1] = w[1] - q;
  } else {
    const long long qx = -((w[5] - w[3]) >> 3), qy = -((w[7] - w[1]) >> 3);
    const long long q2 = (((w[8] - w[6]) - w[2]) + w[0]) >> 6;
    const long long a = w[4] + qx, b = w[4] - qx;
    const long long s = cross_sign > 0 ? q2 : -q2;
    pr[0] = a + qy + s;
    pr[1] = b + qy - s;
    pr[2] = a - qy - s;
    pr[3] = b - qy + s;
  }
#pragma unroll
  for (int ci = 0; ci < (1 << D); ++ci) {
    long long d = half_units30(hc[ci]) - pr[ci];
    d = d < 0 ? -d : d;
    imax = d > imax ? d : imax;
  }
  return true;
}

// 2D and 1D: at most 80 registers, 3 blocks per SM (the stencil-sharing
// barriers of one block are covered by the others); 3D: 2 blocks, 128
// registers (with a minimum of one block the compiler takes 150)
template <int D, int Q, int F>
__global__ void __launch_bounds__(256, D == 3 ? 2 : 3) k_details(const InstDev* __restrict__ IB, int n, int cur) {
  using S = typename FormT<F>::S;
  constexpr int PY = PopRows<Q>::value;
  extern __shared__ int pre[];
  __shared__ InstDev si;
  // the group norm is a maximum of absolute values: compared as the integer
  // bit patterns of non-negative doubles (same order), on the integer pipe
  __shared__ unsigned long long red[PY][32];
  // the cell's 3^D stencil entries and 2^D child entries, looked up once per
  // cell (spread over the population rows) and shared through the block
  constexpr int NS = Pow3<D>::value, NE = NS + (1 << D);
  __shared__ int32_t sent[NE][32];
  int have = -1;
  mr_inst_prefetch(si, have, IB, n);
  mr_grid_dep();  // after the copy of the descriptor, which no step kernel writes
  const int tiles = mr_group_prefix(pre, n, [&](int b) { return (IB[b].mesh[cur].cnt->total[MR_CLS_INT] + 31) / 32; });
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {  // uniform over the block
    const int b = mr_group_find(pre, n, t);
    mr_inst_use(si, have, IB, b);
    const Geo& g = si.g;
    const MeshDev& A = si.mesh[cur];
    const void* LF = si.fstate;
    const int nI = A.cnt->total[MR_CLS_INT];
    const int i = (t - pre[b]) * 32 + threadIdx.x;
    if (i < nI) {
      const int L = A.lvl[MR_CLS_INT][i];
      const uint32_t code = A.code[MR_CLS_INT][i];
      int c[3] = {0, 0, 0};
      mr_decode_d<D>(g, L, code, c);
      for (int e = threadIdx.y; e < NE; e += PY)
        sent[e][threadIdx.x] = e < NS ? mr_stencil_entry_d<D>(g, A, L, c, e)
                                      : A.map[g.base[L + 1] + ((code << D) | (uint32_t)(e - NS))];
    }
    __syncthreads();
    unsigned long long gmax = 0ull;
    if (i < nI) {
      bool ok = true;
      ValPtr<S> sv[NS], cv[1 << D];
#pragma unroll
      for (int kk = 0; kk < NS; ++kk) {
        const int32_t e = sent[kk][threadIdx.x];
        ok = ok && (((uint32_t)e) >> 30) <= MR_CLS_INT;
        sv[kk] = mr_resolve<S>(g, A, LF, e);
      }
#pragma unroll
      for (int ci = 0; ci < (1 << D); ++ci) {
        const int32_t e = sent[NS + ci][threadIdx.x];
        ok = ok && e != MR_MAP_NONE && (((uint32_t)e) >> 30) <= MR_CLS_INT;
        cv[ci] = mr_resolve<S>(g, A, LF, e);
      }
      if (!ok) {
        if (threadIdx.y == 0) mr_set_err(A.cnt, MR_DERR_INTERNAL);
      } else {
        long long imax = 0;  // FP16 storage: largest |detail| in units of 2^-30
#pragma unroll
        for (int p = threadIdx.y; p < Q; p += PY) {
          if constexpr (F == MR_FORM_F32_F16) {
            if (half_details<D>(sv, cv, p, g.cross_sign, imax)) continue;
          }
          double v[NS], c[1 << D];
#pragma unroll
          for (int kk = 0; kk < NS; ++kk) v[kk] = mr_ld(sv[kk], p);
#pragma unroll
          for (int ci = 0; ci < (1 << D); ++ci) c[ci] = mr_ld(cv[ci], p);
          double pr[1 << D];
          mr_predict_children_canonical<D>(v, g.cross_sign, pr);
#pragma unroll
          for (int ci = 0; ci < (1 << D); ++ci) {
            const unsigned long long a =
                (unsigned long long)__double_as_longlong(__dsub_rn(c[ci], pr[ci])) & 0x7fffffffffffffffull;
            gmax = a > gmax ? a : gmax;
          }
        }
        if (imax > 0) {
          // exact: imax < 2^50, and the scaling is a power of two
          const unsigned long long a =
              (unsigned long long)__double_as_longlong(__dmul_rn(__ll2double_rn(imax), 0x1p-30));
          gmax = a > gmax ? a : gmax;
        }
      }
    }
    red[threadIdx.y][threadIdx.x] = gmax;
    __syncthreads();
    if (threadIdx.y == 0 && i < nI) {
      unsigned long long mb = red[0][threadIdx.x];
#pragma unroll
      for (int kk = 1; kk < PY; ++kk) mb = red[kk][threadIdx.x] > mb ? red[kk][threadIdx.x] : mb;
      const double m = __longlong_as_double((long long)mb);
      A.G[i] = m;
    }
    __syncthreads();
  }
}

template <int D, int Q, int F>
void launch_project_t(const Group& G, int cur, int k, cudaStream_t st) {
  mr_launch_pdl(k_project<D, Q, F>, mr_tile_grid(G, G.proj_cells[k], 32, G.bps[MR_PH_PROJECT]), dim3(32, PopRows<Q>::value),
                mr_pre_bytes(G), st, G.dev, G.n, cur, k);
}
template <int D, int Q, int F>
void launch_details_t(const Group& G, int cur, cudaStream_t st) {
  mr_launch_pdl(k_details<D, Q, F>, mr_tile_grid(G, G.capI, 32, G.bps[MR_PH_DETAILS]), dim3(32, PopRows<Q>::value), mr_pre_bytes(G),
                st, G.dev, G.n, cur);
}

}  // namespace

#define MR_DISPATCH_F(FN, D, Q, ...)                       \
  switch (G.form) {                                        \
    case MR_FORM_F64: FN<D, Q, MR_FORM_F64>(__VA_ARGS__); break;       \
    case MR_FORM_F32: FN<D, Q, MR_FORM_F32>(__VA_ARGS__); break;       \
    case MR_FORM_F32_F16: FN<D, Q, MR_FORM_F32_F16>(__VA_ARGS__); break; \
    case MR_FORM_F32_BF16: FN<D, Q, MR_FORM_F32_BF16>(__VA_ARGS__); break; \
  }

#define MR_DISPATCH_DQF(FN, ...)                                  \
  switch (G.d * 100 + G.Q) {                                      \
    case 102: MR_DISPATCH_F(FN, 1, 2, __VA_ARGS__); break;        \
    case 103: MR_DISPATCH_F(FN, 1, 3, __VA_ARGS__); break;        \
    case 209: MR_DISPATCH_F(FN, 2, 9, __VA_ARGS__); break;        \
    case 216: MR_DISPATCH_F(FN, 2, 16, __VA_ARGS__); break;       \
    case 306: MR_DISPATCH_F(FN, 3, 6, __VA_ARGS__); break;        \
    default: break;                                               \
  }

void mr_launch_project(const Group& G, int cur, int k, cudaStream_t st) {
  MR_DISPATCH_DQF(launch_project_t, G, cur, k, st);
}

void mr_launch_details(const Group& G, int cur, cudaStream_t st) {
  if (G.s > 1) return mr_launch_details_w(G, cur, st);
  MR_DISPATCH_DQF(launch_details_t, G, cur, st);
}

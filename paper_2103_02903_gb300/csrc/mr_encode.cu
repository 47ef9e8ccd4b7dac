// Multiresolution encode of the stored field (Sec. 4.1-4.2): bottom-up
// projection of the leaves into the internal cells of R(Lambda)
// (Def. Projection) and the details of every cell of R(Lambda) above J_min
// reduced to one max-norm per sibling group and over all populations
// (Def. Details and the group norm of Sec. 4.4).
//
// Both kernels evaluate their arithmetic in a fixed order with
// __dadd_rn/__dmul_rn (never contracted into FMA), so that the details, and
// hence every keep / refine decision, carry the same bits as the CPU oracle
// on the same leaf values.
#include "mr_common.cuh"

namespace {

template <int D, int Q>
__global__ void __launch_bounds__(256) k_project(Geo g, MeshDev A, const double* __restrict__ LF,
                                                 int level) {
  const int begin = A.cnt->off[MR_CLS_INT][level], end = A.cnt->off[MR_CLS_INT][level + 1];
  const double scale = D == 1 ? 0.5 : 0.25;
  for (int i = begin + blockIdx.x * blockDim.x + threadIdx.x; i < end; i += gridDim.x * blockDim.x) {
    const uint32_t code = A.code[MR_CLS_INT][i];
    ValPtr ch[1 << D];
    bool ok = true;
#pragma unroll
    for (int ci = 0; ci < (1 << D); ++ci) {
      int32_t e = A.map[g.base[level + 1] + ((code << D) | (uint32_t)ci)];
      ok = ok && e != MR_MAP_NONE && (((uint32_t)e) >> 30) <= MR_CLS_INT;
      ch[ci] = mr_resolve(g, A, LF, e);
    }
    if (!ok) {
      mr_set_err(A.cnt, MR_DERR_INTERNAL);
      continue;
    }
#pragma unroll 4
    for (int p = 0; p < Q; ++p) {
      double acc = 0.0;
#pragma unroll
      for (int ci = 0; ci < (1 << D); ++ci) acc = __dadd_rn(acc, mr_ld(ch[ci], p));
      A.IF[(size_t)p * g.cap[1] + i] = __dmul_rn(acc, scale);
    }
  }
}

template <int D, int Q>
__global__ void __launch_bounds__(256) k_details(Geo g, MeshDev A, const double* __restrict__ LF) {
  const int n = A.cnt->total[MR_CLS_INT];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int L = A.lvl[MR_CLS_INT][i];
    const uint32_t code = A.code[MR_CLS_INT][i];
    int x, y;
    mr_decode(g, L, code, x, y);
    int32_t st[9];
    bool ok = mr_stencil_entries<D>(g, A, L, x, y, st);
    ValPtr sv[D == 2 ? 9 : 3], cv[1 << D];
#pragma unroll
    for (int k = 0; k < (D == 2 ? 9 : 3); ++k) {
      ok = ok && (((uint32_t)st[k]) >> 30) <= MR_CLS_INT;
      sv[k] = mr_resolve(g, A, LF, st[k]);
    }
#pragma unroll
    for (int ci = 0; ci < (1 << D); ++ci) {
      int32_t e = A.map[g.base[L + 1] + ((code << D) | (uint32_t)ci)];
      ok = ok && e != MR_MAP_NONE && (((uint32_t)e) >> 30) <= MR_CLS_INT;
      cv[ci] = mr_resolve(g, A, LF, e);
    }
    if (!ok) {
      mr_set_err(A.cnt, MR_DERR_INTERNAL);
      A.G[i] = 0.0;
      continue;
    }
    double gmax = 0.0;
    for (int p = 0; p < Q; ++p) {
      double v[D == 2 ? 9 : 3];
#pragma unroll
      for (int k = 0; k < (D == 2 ? 9 : 3); ++k) v[k] = mr_ld(sv[k], p);
#pragma unroll
      for (int ci = 0; ci < (1 << D); ++ci) {
        double det = __dsub_rn(mr_ld(cv[ci], p), mr_predict_canonical<D>(v, ci, g.cross_sign));
        gmax = fmax(gmax, fabs(det));
      }
    }
    A.G[i] = gmax;
  }
}

template <int D, int Q>
void launch_project_t(const Geo& g, const MeshDev& A, const double* LF, int level, cudaStream_t st,
                      int grid) {
  k_project<D, Q><<<grid, 256, 0, st>>>(g, A, LF, level);
}
template <int D, int Q>
void launch_details_t(const Geo& g, const MeshDev& A, const double* LF, cudaStream_t st, int grid) {
  k_details<D, Q><<<grid, 256, 0, st>>>(g, A, LF);
}

}  // namespace

#define MR_DISPATCH_DQ(FN, ...)                                  \
  switch (g.d * 100 + g.Q) {                                     \
    case 102: FN<1, 2>(__VA_ARGS__); break;                      \
    case 103: FN<1, 3>(__VA_ARGS__); break;                      \
    case 216: FN<2, 16>(__VA_ARGS__); break;                     \
    case 209: FN<2, 9>(__VA_ARGS__); break;                      \
    default: break;                                              \
  }

void mr_launch_project(const Geo& g, const MeshDev& A, const double* LF, int level, cudaStream_t st,
                       int grid) {
  MR_DISPATCH_DQ(launch_project_t, g, A, LF, level, st, grid);
}

void mr_launch_details(const Geo& g, const MeshDev& A, const double* LF, cudaStream_t st, int grid) {
  MR_DISPATCH_DQ(launch_details_t, g, A, LF, st, grid);
}

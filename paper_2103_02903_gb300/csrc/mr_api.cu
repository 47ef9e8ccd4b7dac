// C-ABI of the GB300 adaptive MR-LBM library (declared in include/mr_lbm.h):
// handle life cycle, the host-side flattened-weight tables of
// Eq. PredictionWithMatrixNew, and the orchestration of one time step of
// Algorithm 1 as a fixed sequence of kernels on the handle's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "mr_handle.cuh"

namespace {

mr_status fail(mr_lbm* h, mr_status s) {
  if (h && h->sticky == MR_OK) h->sticky = s;
  return s;
}

bool cuda_ok(mr_lbm* h, cudaError_t e) {
  if (e != cudaSuccess) {
    fail(h, MR_ECUDA);
    return false;
  }
  return true;
}

template <class T>
bool dalloc(mr_lbm* h, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    *p = nullptr;
    return false;
  }
  h->allocs.push_back(q);
  *p = (T*)q;
  return true;
}

// ----------------------------------------------------------------- geometry
bool scheme_setup(Geo& g, const mr_lbm_config* c) {
  memset(g.eta, 0, sizeof(g.eta));
  memset(g.consw, 0, sizeof(g.consw));
  const double L = c->lambda;
  switch (c->scheme) {
    case MR_D1Q2_ADVECTION:
    case MR_D1Q2_BURGERS:
      g.d = 1; g.q = 2; g.m = 1; g.ncons = 1;
      g.eta[0][0] = 1; g.eta[1][0] = -1;
      g.opp[0] = 1; g.opp[1] = 0;
      g.consw[0][0] = 1; g.consw[0][1] = 1;
      break;
    case MR_D1Q3_SHALLOW_WATER:
      g.d = 1; g.q = 3; g.m = 1; g.ncons = 2;
      g.eta[1][0] = 1; g.eta[2][0] = -1;
      g.opp[0] = 0; g.opp[1] = 2; g.opp[2] = 1;
      g.consw[0][0] = g.consw[0][1] = g.consw[0][2] = 1;
      g.consw[1][1] = L; g.consw[1][2] = -L;
      break;
    case MR_D2Q4x4_EULER:
      g.d = 2; g.q = 4; g.m = 4; g.ncons = 4;
      g.eta[0][0] = 1; g.eta[1][1] = 1; g.eta[2][0] = -1; g.eta[3][1] = -1;
      g.opp[0] = 2; g.opp[1] = 3; g.opp[2] = 0; g.opp[3] = 1;
      for (int i = 0; i < 4; ++i)
        for (int h = 0; h < 4; ++h) g.consw[i][4 * i + h] = 1;
      break;
    case MR_D2Q9_NS: {
      static const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
      static const int op[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
      g.d = 2; g.q = 9; g.m = 1; g.ncons = 3;
      for (int h = 0; h < 9; ++h) {
        g.eta[h][0] = ex[h];
        g.eta[h][1] = ey[h];
        g.opp[h] = op[h];
        g.consw[0][h] = 1;
        g.consw[1][h] = L * ex[h];
        g.consw[2][h] = L * ey[h];
      }
      break;
    }
    case MR_D3Q6_ADVECTION:
      g.d = 3; g.q = 6; g.m = 1; g.ncons = 1;
      for (int h = 0; h < 6; ++h) {
        g.eta[h][h / 2] = (h & 1) ? -1 : 1;
        g.opp[h] = h ^ 1;
        g.consw[0][h] = 1;
      }
      break;
    default:
      return false;
  }
  g.Q = g.q * g.m;
  return true;
}

// One-dimensional reconstruction (prediction with s = 1 applied `gap`
// times) of a level field of N cells, constant extension or wrap outside.
void recon1d(std::vector<double>& cur, int N, int gap, bool periodic) {
  for (int it = 0; it < gap; ++it) {
    std::vector<double> nxt(2 * (size_t)N);
    for (int k = 0; k < N; ++k) {
      auto at = [&](int i) {
        if (periodic) return cur[((i % N) + N) % N];
        return cur[std::min(std::max(i, 0), N - 1)];
      };
      const double q = -0.125 * (at(k + 1) - at(k - 1));
      nxt[2 * k] = cur[k] + q;
      nxt[2 * k + 1] = cur[k] - q;
    }
    cur.swap(nxt);
    N *= 2;
  }
}

// Flattened weights (Eq. PredictionWithMatrixNew) of one axis: for a cell k
// of a level with N cells and `gap` levels above the finest, the weights of
// f_{k+delta}, delta = -2..2, in the finest edge values R_{k-1}, R_k, L_k,
// L_{k+1}.  out[0..4] = R_{k-1} - R_k (incoming minus outgoing for the
// velocity +1; R_{k-1} left out at a non-periodic left boundary),
// out[5..9] = L_{k+1} - L_k (velocity -1), out[10..14] = R_k, out[15..19] = L_k.
bool axis_weights(int N, int gap, bool periodic, int k, double* out) {
  int Nsim = N, ks = k;
  if (periodic) {  // interior weights, computed away from any boundary
    Nsim = 9;
    ks = 4;
  }
  const int n = 1 << gap;
  for (int dl = -2; dl <= 2; ++dl) {
    const int i = ks + dl;
    double r0 = 0, r1 = 0, l0 = 0, l1 = 0;
    if (i >= 0 && i < Nsim) {
      std::vector<double> f(Nsim, 0.0);
      f[i] = 1.0;
      recon1d(f, Nsim, gap, false);
      if (ks >= 1) r0 = f[(size_t)n * ks - 1];
      r1 = f[(size_t)n * (ks + 1) - 1];
      l0 = f[(size_t)n * ks];
      if (ks + 1 < Nsim) l1 = f[(size_t)n * (ks + 1)];
    } else if (!periodic) {
      // outside the domain: the kernel never reads it, the weight must be 0
    }
    out[dl + 2] = r0 - r1;
    out[5 + dl + 2] = l1 - l0;
    out[10 + dl + 2] = r1;
    out[15 + dl + 2] = l0;
  }
  return true;
}

// The same four tables for the prediction of half-width s = 2, 3, over the
// window delta = -W..W (W = 2s) of the slot layout of mr_slot_w:
// out[t * (2W + 1) + delta + W], t as in axis_weights.
// Table 1: c_1 .. c_s of the prediction of half-width s.
const double kPredCoef[4][3] = {
    {0.0, 0.0, 0.0},
    {-1.0 / 8.0, 0.0, 0.0},
    {-22.0 / 128.0, 3.0 / 128.0, 0.0},
    {-201.0 / 1024.0, 11.0 / 256.0, -5.0 / 1024.0},
};

// One-dimensional reconstruction with the prediction of half-width s applied
// `gap` times to a level field of N cells, constant extension outside.
void recon1d_s(std::vector<double>& cur, int N, int gap, int s) {
  for (int it = 0; it < gap; ++it) {
    std::vector<double> nxt(2 * (size_t)N);
    auto at = [&](int i) { return cur[std::min(std::max(i, 0), N - 1)]; };
    for (int k = 0; k < N; ++k) {
      double q = 0.0;
      for (int a = 1; a <= s; ++a) q += kPredCoef[s][a - 1] * (at(k + a) - at(k - a));
      nxt[2 * k] = cur[k] + q;
      nxt[2 * k + 1] = cur[k] - q;
    }
    cur.swap(nxt);
    N *= 2;
  }
}

void axis_weights_w(int N, int gap, bool periodic, int k, int s, int W, double* out) {
  const int NW = 2 * W + 1;
  int Nsim = N, ks = k;
  if (periodic) {  // interior weights, computed away from any face of the patch
    Nsim = 4 * W + 5;
    ks = 2 * W + 2;
  }
  const size_t n = (size_t)1 << gap;
  for (int dl = -W; dl <= W; ++dl) {
    const int i = ks + dl;
    double r0 = 0, r1 = 0, l0 = 0, l1 = 0;
    if (i >= 0 && i < Nsim) {  // outside a non-periodic domain the kernel reads nothing: weight 0
      std::vector<double> f(Nsim, 0.0);
      f[i] = 1.0;
      recon1d_s(f, Nsim, gap, s);
      if (ks >= 1) r0 = f[n * ks - 1];
      r1 = f[n * (ks + 1) - 1];
      l0 = f[n * ks];
      if (ks + 1 < Nsim) l1 = f[n * (ks + 1)];
    }
    out[0 * NW + dl + W] = r0 - r1;
    out[1 * NW + dl + W] = l1 - l0;
    out[2 * NW + dl + W] = r1;
    out[3 * NW + dl + W] = l0;
  }
}

void build_tables_w(const Geo& g, std::vector<double>& Ws) {
  const int W = 2 * g.s_pred, NW = 2 * W + 1;
  Ws.assign((size_t)MR_WWIDX(g.J + 1, 0, 0, 0, W), 0.0);
  std::vector<double> w(4 * NW);
  for (int l = g.Jmin; l <= g.J; ++l)
    for (int a = 0; a < g.d; ++a) {
      const int N = g.n[l][a];
      const bool per = g.periodic[a] != 0;
      std::vector<int> ks;
      if (per) {
        ks.push_back(0);
      } else if (N <= NW) {
        for (int k = 0; k < N; ++k) ks.push_back(k);
      } else {
        for (int k = 0; k <= W; ++k) ks.push_back(k);
        for (int k = N - W; k < N; ++k) ks.push_back(k);
      }
      for (int k : ks) {
        const int sl = mr_slot_w(k, N, per, W);
        axis_weights_w(N, g.J - l, per, k, g.s_pred, W, w.data());
        for (int t = 0; t < MR_NTAB; ++t)
          for (int e = 0; e < NW; ++e) Ws[MR_WWIDX(l, a, sl, t, W) + e] = w[t * NW + e];
      }
    }
}

void build_tables(const Geo& g, std::vector<double>& W) {
  W.assign((size_t)(g.J + 1) * 3 * MR_NSLOT * MR_NTAB * 5, 0.0);
  for (int l = g.Jmin; l <= g.J; ++l)
    for (int a = 0; a < g.d; ++a) {
      const int N = g.n[l][a];
      const bool per = g.periodic[a] != 0;
      for (int s = 0; s < MR_NSLOT; ++s) {
        int k;
        if (per) {
          if (s != 2) continue;
          k = 2;
        } else {
          k = s < 2 ? s : (s == 2 ? 2 : N - 2 + (s - 3));
          if (k < 0 || k >= N || mr_slot(k, N, 0) != s) continue;
        }
        double w[20];
        axis_weights(N, g.J - l, per, k, w);
        for (int t = 0; t < MR_NTAB; ++t)
          for (int e = 0; e < 5; ++e) W[MR_WIDX(l, a, s, t) + e] = w[t * 5 + e];
      }
    }
}

// Equilibrium populations M^{-1} m^eq(u) of each scheme on the host (used for
// the storage offsets of the 16-bit forms).
void host_equilibrium(const Geo& g, const double* u, double* f) {
  const double L = g.lambda;
  switch (g.scheme) {
    case MR_D1Q2_ADVECTION:
    case MR_D1Q2_BURGERS: {
      const double m1 = g.scheme == MR_D1Q2_ADVECTION ? g.phys[0] * u[0] : 0.5 * u[0] * u[0];
      f[0] = 0.5 * (u[0] + m1 / L);
      f[1] = 0.5 * (u[0] - m1 / L);
      break;
    }
    case MR_D1Q3_SHALLOW_WATER: {
      const double t = (u[1] * u[1] / u[0] + 0.5 * g.phys[0] * u[0] * u[0]) / (L * L);
      f[0] = u[0] - t;
      f[1] = 0.5 * (t + u[1] / L);
      f[2] = 0.5 * (t - u[1] / L);
      break;
    }
    case MR_D2Q4x4_EULER: {
      const double rho = u[0], mx = u[1], my = u[2], E = u[3];
      const double vx = mx / rho, vy = my / rho;
      const double pr = (g.phys[0] - 1.0) * (E - 0.5 * (mx * vx + my * vy));
      const double fx[4] = {mx, mx * vx + pr, my * vx, vx * (E + pr)};
      const double fy[4] = {my, mx * vy, my * vy + pr, vy * (E + pr)};
      for (int i = 0; i < 4; ++i) {
        const double a = 0.25 * u[i], b = 0.5 * fx[i] / L, c = 0.5 * fy[i] / L;
        f[4 * i + 0] = a + b;
        f[4 * i + 1] = a + c;
        f[4 * i + 2] = a - b;
        f[4 * i + 3] = a - c;
      }
      break;
    }
    case MR_D3Q6_ADVECTION: {
      // m^eq = (u, V u, 0, 0): a = b = c = u / 3 (see Scheme<5>)
      const double a = u[0] / 3.0;
      for (int h = 0; h < 6; ++h) f[h] = 0.5 * (a + ((h & 1) ? -1.0 : 1.0) * g.phys[h / 2] * u[0] / L);
      break;
    }
    case MR_D2Q9_NS: {
      // orthogonal integer rows R_r (the rows of M over their power of
      // lambda): f = sum_r R_r mu_r / |R_r|^2, j = q / lambda
      static const int R[9][9] = {{1, 1, 1, 1, 1, 1, 1, 1, 1},         {0, 1, 0, -1, 0, 1, -1, -1, 1},
                                  {0, 0, 1, 0, -1, 1, 1, -1, -1},      {-4, -1, -1, -1, -1, 2, 2, 2, 2},
                                  {0, -2, 0, 2, 0, 1, -1, -1, 1},      {0, 0, -2, 0, 2, 1, 1, -1, -1},
                                  {4, -2, -2, -2, -2, 1, 1, 1, 1},     {0, 1, -1, 1, -1, 0, 0, 0, 0},
                                  {0, 0, 0, 0, 0, 1, -1, 1, -1}};
      const double rho = u[0], jx = u[1] / L, jy = u[2] / L;
      const double j2 = (jx * jx + jy * jy) / rho;
      const double mu[9] = {rho, jx, jy, -2.0 * rho + 3.0 * j2, -jx, -jy, rho - 3.0 * j2,
                            (jx * jx - jy * jy) / rho, jx * jy / rho};
      for (int h = 0; h < 9; ++h) {
        double acc = 0.0;
        for (int r = 0; r < 9; ++r) {
          double n2 = 0.0;
          for (int k = 0; k < 9; ++k) n2 += (double)(R[r][k] * R[r][k]);
          acc += R[r][h] * mu[r] / n2;
        }
        f[h] = acc;
      }
      break;
    }
  }
}

mr_status validate(const mr_lbm_config* c) {
  if (!c) return MR_EINVAL;
  if (c->scheme < 0 || c->scheme > MR_D3Q6_ADVECTION) return MR_EINVAL;
  if (c->scheme == MR_D3Q6_ADVECTION && c->max_level > 10) return MR_EINVAL;  // 30-bit 3-way codes
  if (c->scheme == MR_D2Q9_NS && c->cross_sign == -1) return MR_EINVAL;  // needs the tensor product
  if (c->obstacle != 0 && (c->obstacle != 1 || c->scheme != MR_D2Q9_NS)) return MR_EINVAL;
  for (int f = 0; f < 6; ++f)
    if (c->bc[f] == MR_BC_BOUNCE_BACK_VELOCITY && c->scheme != MR_D2Q9_NS) return MR_EINVAL;
  if (c->obstacle && !(c->xmax[0] > c->xmin[0]) ) return MR_EINVAL;
  if (!(c->lambda > 0) || !(c->eps >= 0) || c->mu_bar < 0) return MR_EINVAL;
  if (c->pred_s < 0 || c->pred_s > 3) return MR_EINVAL;
  const int s_pred = c->pred_s ? c->pred_s : 1;
  if (c->mu_bar > 2 * s_pred + 1) return MR_EINVAL;  // the regularity guess lies in [0, 2s + 1] (Sec. 5.1)
  if (c->precision < MR_FP64 || c->precision > MR_FP32_BF16STORE) return MR_EINVAL;
  if (c->min_level < 2 || c->max_level < c->min_level || c->max_level > 15) return MR_EINVAL;
  for (int i = 0; i < 16; ++i)
    if (!(c->s[i] >= 0.0 && c->s[i] <= 2.0)) return MR_EINVAL;
  for (int f = 0; f < 6; ++f)
    if (c->bc[f] < MR_BC_PERIODIC || c->bc[f] > MR_BC_BOUNCE_BACK_VELOCITY) return MR_EINVAL;
  for (int a = 0; a < 3; ++a)
    if ((c->bc[2 * a] == MR_BC_PERIODIC) != (c->bc[2 * a + 1] == MR_BC_PERIODIC)) return MR_EINVAL;
  if (c->cross_sign != 0 && c->cross_sign != 1 && c->cross_sign != -1) return MR_EINVAL;
  if (c->exact_collision != 0 &&
      (c->exact_collision != 1 || c->precision != MR_FP64 || c->scheme == MR_D3Q6_ADVECTION))
    return MR_EINVAL;
  return MR_OK;
}

int grid_for(const mr_lbm* h, int per_sm = 4) { return h->nsm * per_sm; }

void count_launch(mr_lbm* h, int n = 1) { h->launches += n; }

mr_status check_launch(mr_lbm* h) {
  if (cudaGetLastError() != cudaSuccess) return fail(h, MR_ECUDA);
  return MR_OK;
}

mr_status read_counts(mr_lbm* h, MeshCounts* out /*[2]*/) {
  if (!cuda_ok(h, cudaMemcpyAsync(out, h->cntbuf, 2 * sizeof(MeshCounts), cudaMemcpyDeviceToHost, h->st)))
    return MR_ECUDA;
  if (!cuda_ok(h, cudaStreamSynchronize(h->st))) return MR_ECUDA;
  const int err = out[0].err | out[1].err;
  if (err & MR_DERR_CAPACITY) return fail(h, MR_ECAPACITY);
  if (err & MR_DERR_INPUT) return fail(h, MR_EINVAL);
  if (err & MR_DERR_INTERNAL) return fail(h, MR_EINTERNAL);
  if (err & MR_DERR_NONFINITE) return fail(h, MR_ENONFINITE);
  return MR_OK;
}

// ----------------------------------------------------------------- groups
void fill_desc(const mr_lbm* h, InstDev& d) {
  memset(&d, 0, sizeof(d));
  d.g = h->g;
  d.mesh[0] = h->mesh[0];
  d.mesh[1] = h->mesh[1];
  d.fstate = h->fstate;
  d.fscratch = h->fscratch;
  d.flags = h->flags;
  d.cls = h->cls;
  d.act = h->act;
  d.acth = h->act + h->g.base[h->g.J + 1] / MR_DENSE_ALIGN;
  d.bcounts = h->bcounts;
  d.W = h->W;
  d.Wf = h->Wf;
  d.det = h->det;
  d.Ws = h->Ws;
  d.Wsf = h->Wsf;
  auto& k = d.g.f32;  // FP32 copies for the FP32 arithmetic of the forms
  k.lambda = (float)d.g.lambda;
  k.inv_lambda = (float)d.g.inv_lambda;
  k.cross_sign = (float)d.g.cross_sign;
  for (int i = 0; i < 16; ++i) k.s[i] = (float)d.g.s[i];
  for (int i = 0; i < 8; ++i) k.phys[i] = (float)d.g.phys[i];
  for (int p = 0; p < MR_MAXQ; ++p) {
    k.off[p] = (float)d.g.off[p];
    k.feq0[p] = (float)d.g.feq0[p];
    k.bcv[p] = (float)d.g.bcv[p];
  }
}

// Write the handle's descriptor to its device slot (stream-ordered).
bool upload_desc(mr_lbm* h) {
  InstDev d;
  fill_desc(h, d);
  return cuda_ok(h, cudaMemcpyAsync(h->dinst, &d, sizeof(d), cudaMemcpyHostToDevice, h->st));
}

// Host summary of a group whose descriptors are at `dev`; chunk_pre[n + 1]
// is written to `dchunk` on stream st.
bool make_group(Group& G, const std::vector<const mr_lbm*>& members, const InstDev* dev, int* dchunk,
                cudaStream_t st, int nsm) {
  memset(&G, 0, sizeof(G));
  G.dev = dev;
  G.chunk_pre = dchunk;
  G.n = (int)members.size();
  G.nsm = nsm;
  const Geo& g0 = members[0]->g;
  G.d = g0.d;
  G.Q = g0.Q;
  G.scheme = g0.scheme;
  G.form = g0.form;
  G.s = g0.s_pred;
  {
    const int def[MR_NPH] = MR_DEFAULT_BPS;
    for (int ph = 0; ph < MR_NPH; ++ph) G.bps[ph] = def[ph];
  }
  std::vector<int> pre(G.n + 1, 0);
  for (int b = 0; b < G.n; ++b) {
    const Geo& g = members[b]->g;
    const int chunks = (int)(g.base[g.J + 1] / MR_DENSE_ALIGN);
    pre[b + 1] = pre[b] + chunks;
    G.span = std::max(G.span, g.J - g.Jmin);
    G.grade = G.grade || g.J > g.Jmin + 1;
    G.capL += g.cap[0];
    G.capI += g.cap[1];
    for (int k = 1; k <= g.J - g.Jmin; ++k) {
      G.proj_cells[k] += g.ncode[g.J - k];
      G.pred_cells[k] += g.ncode[g.Jmin + k];
    }
  }
  G.chunks = pre[G.n];
  return cudaMemcpyAsync(dchunk, pre.data(), pre.size() * sizeof(int), cudaMemcpyHostToDevice, st) == cudaSuccess &&
         cudaStreamSynchronize(st) == cudaSuccess;
}

// ----------------------------------------------------------------- execution
cudaEvent_t next_event(Exec& x) {
  if (x.ev_used == x.ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    x.ev_pool.push_back(e);
  }
  return x.ev_pool[x.ev_used++];
}

// Kernel groups that the profile calls can time.
enum { PG_STREAM = 1, PG_DETAILS = 2, PG_PROJECT = 3, PG_PREDICT = 4, PG_MESH = 5, PG_REMESH = 6 };

inline void prof_begin(Exec& x, int group) {
  if (x.prof_group == group) cudaEventRecord(next_event(x), x.st);
}
inline void prof_end(Exec& x, int group) {
  if (x.prof_group == group) cudaEventRecord(next_event(x), x.st);
}

// Encode of the current state: internal values, bottom-up (Def. Projection).
void run_projection(Exec& x, const Group& G, int cur) {
  for (int k = 1; k <= G.span; ++k) {
    prof_begin(x, PG_PROJECT);
    mr_launch_project(G, cur, k, x.st);
    prof_end(x, PG_PROJECT);
    x.launches += 1;
  }
}

// Build mesh `dst` from the classification in cls (LEAF / INT bits).
void run_build(Exec& x, const Group& G, int dst) {
  mr_launch_mark_ghosts(G, x.st);
  mr_launch_compact(G, dst, x.st);
  x.launches += 4;
}

// Adaptation and data transfer; on return the new mesh is 1 - cur and its
// (pre-transport) leaf values are in fscratch.
void run_adapt(Exec& x, const Group& G, int cur) {
  run_projection(x, G, cur);
  prof_begin(x, PG_DETAILS);
  mr_launch_details(G, cur, x.st);
  prof_end(x, PG_DETAILS);
  prof_begin(x, PG_MESH);
  mr_launch_flags_T(G, cur, x.st);
  mr_launch_flags_H(G, cur, x.st);
  mr_launch_grade(G, x.st);
  mr_launch_classify(G, x.st);
  x.launches += G.grade ? 5 : 4;
  run_build(x, G, 1 - cur);
  prof_end(x, PG_MESH);
  prof_begin(x, PG_REMESH);
  mr_launch_remesh_copy(G, cur, x.st);
  prof_end(x, PG_REMESH);
  x.launches += 1;
  for (int k = 1; k <= G.span; ++k) {
    prof_begin(x, PG_PREDICT);
    mr_launch_predict_level(G, 1 - cur, k, x.st);
    prof_end(x, PG_PREDICT);
    x.launches += 1;
  }
}

void run_stream(Exec& x, const Group& G, int dst, int do_stream, int do_collide) {
  prof_begin(x, PG_STREAM);
  if (do_stream && G.s > 1) {
    mr_launch_edge_details_w(G, dst, x.st);  // the critical-case details, once per refined cell
    x.launches += 1;
  } else if (do_stream && G.scheme == MR_D2Q9_NS) {
    mr_launch_edge_details(G, dst, x.st);
    x.launches += 1;
  }
  mr_launch_stream_collide(G, dst, do_stream, do_collide, x.st, 1);  // counts the step
  prof_end(x, PG_STREAM);
  x.launches += 1;
}

// One iteration of the loop of Algorithm 1 for every instance of a group.
void run_step(Exec& x, const Group& G, int cur) {
  run_adapt(x, G, cur);
  run_stream(x, G, 1 - cur, 1, G.exact ? 0 : 1);
  if (G.exact) x.launches += mr_launch_exact_collision(G, 1 - cur, G.exact, G.exact_nd, x.st);
}

void drop_graphs(Exec& x) {
  for (auto& G : x.graphs) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G.exec = nullptr;
    G.graph = nullptr;
    G.prof = -1;
    G.ev_nodes.clear();
  }
}

// Capture `body` (the launches of one step on x.st) for the current mesh
// parity into x.graphs[x.cur].
template <class Body>
bool capture_step(Exec& x, Body body) {
  StepGraph& G = x.graphs[x.cur];
  if (!x.cap_st && cudaStreamCreateWithFlags(&x.cap_st, cudaStreamNonBlocking) != cudaSuccess) return false;
  while (x.ev_pool.size() < x.ev_used + 64) {  // events are created outside the capture
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return false;
    x.ev_pool.push_back(e);
  }
  const size_t ev0 = x.ev_used;
  const long long l0 = x.launches;
  cudaStream_t orig = x.st;
  x.st = x.cap_st;
  if (cudaStreamBeginCapture(x.cap_st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    x.st = orig;
    return false;
  }
  body();
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(x.cap_st, &graph);
  x.st = orig;
  std::vector<cudaEvent_t> cap_events(x.ev_pool.begin() + ev0, x.ev_pool.begin() + x.ev_used);
  x.ev_used = ev0;
  G.launches = x.launches - l0;
  x.launches = l0;
  if (e != cudaSuccess || !graph) return false;
  size_t n = 0;
  cudaGraphGetNodes(graph, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  if (n) cudaGraphGetNodes(graph, nodes.data(), &n);
  G.ev_nodes.assign(cap_events.size(), nullptr);
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t ev;
    if (cudaGraphEventRecordNodeGetEvent(nd, &ev) != cudaSuccess) continue;
    for (size_t i = 0; i < cap_events.size(); ++i)
      if (cap_events[i] == ev) G.ev_nodes[i] = nd;
  }
  for (cudaGraphNode_t nd : G.ev_nodes)
    if (!nd) {
      cudaGraphDestroy(graph);
      return false;
    }
  if (cudaGraphInstantiate(&G.exec, graph, 0) != cudaSuccess) {
    cudaGraphDestroy(graph);
    G.exec = nullptr;
    return false;
  }
  G.graph = graph;
  G.prof = x.prof_group;
  return true;
}

// One step by graph replay (captured on first use for this parity and
// profiling mode); false if graphs cannot be used, and nothing was queued.
template <class Body>
bool graph_step(Exec& x, Body body) {
  StepGraph& G = x.graphs[x.cur];
  if (G.exec && G.prof != x.prof_group) {
    cudaGraphExecDestroy(G.exec);
    cudaGraphDestroy(G.graph);
    G.exec = nullptr;
    G.graph = nullptr;
  }
  if (!G.exec && !capture_step(x, body)) return false;
  for (cudaGraphNode_t nd : G.ev_nodes)
    if (cudaGraphExecEventRecordNodeSetEvent(G.exec, nd, next_event(x)) != cudaSuccess) return false;
  if (cudaGraphLaunch(G.exec, x.st) != cudaSuccess) return false;
  x.launches += G.launches;
  return true;
}

// `nsteps` steps queued on x (graph replay, or direct launches when graphs
// are unavailable); x.cur flips after each.
template <class Body>
void queue_steps(Exec& x, int nsteps, Body body) {
  for (int it = 0; it < nsteps; ++it) {
    if (!(x.use_graph && graph_step(x, body))) {
      x.use_graph = false;  // graphs unavailable: launch the kernels directly from now on
      body();
    }
    x.cur = 1 - x.cur;
  }
}

mr_status ensure_staging(mr_lbm* h, size_t bytes) {
  if (h->staging_bytes >= bytes) return MR_OK;
  if (h->staging) cudaFree(h->staging);
  h->staging = nullptr;
  h->staging_bytes = 0;
  if (cudaMalloc(&h->staging, bytes) != cudaSuccess) return fail(h, MR_ENOMEM);
  h->staging_bytes = bytes;
  return MR_OK;
}

double profile_total(Exec& x, long long* launches) {
  double tot = 0;
  for (size_t i = 0; i + 1 < x.ev_used; i += 2) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, x.ev_pool[i], x.ev_pool[i + 1]) != cudaSuccess) return -1.0;
    tot += ms;
  }
  if (launches) *launches = (long long)(x.ev_used / 2);
  return tot;
}

}  // namespace

mr_status mr_handle_fail(mr_lbm* h, mr_status s) { return fail(h, s); }
void mr_handle_projection(mr_lbm* h) { run_projection(*h, h->grp, h->cur); }
mr_status mr_handle_read_counts(mr_lbm* h, MeshCounts* out) { return read_counts(h, out); }

// =================================================================== C-ABI

extern "C" {

const char* mr_lbm_strerror(mr_status s) {
  switch (s) {
    case MR_OK: return "MR_OK";
    case MR_EINVAL: return "MR_EINVAL: invalid argument or configuration";
    case MR_ENOMEM: return "MR_ENOMEM: allocation failed";
    case MR_ECUDA: return "MR_ECUDA: CUDA runtime error";
    case MR_ECAPACITY: return "MR_ECAPACITY: capacity exceeded";
    case MR_ENOCONV: return "MR_ENOCONV: no convergence";
    case MR_ENONFINITE: return "MR_ENONFINITE: non-finite value";
    case MR_ESTATE: return "MR_ESTATE: invalid state for this call";
    case MR_EINTERNAL: return "MR_EINTERNAL: mesh invariant violated";
  }
  return "unknown status";
}

mr_status mr_lbm_flattened_weights(int roots, int level, int max_level, int periodic, int k, double* out) {
  if (!out || roots < 1 || level < 0 || max_level < level || max_level > 20) return MR_EINVAL;
  const int N = roots << level;
  if (k < 0 || k >= N) return MR_EINVAL;
  double w[20];
  int kk = k;
  if (!periodic) {
    const int s = mr_slot(k, N, 0);
    kk = s < 2 ? s : (s == 2 ? k : N - 2 + (s - 3));
  }
  axis_weights(N, max_level - level, periodic != 0, kk, w);
  for (int i = 0; i < 10; ++i) out[i] = w[i];
  return MR_OK;
}

mr_status mr_lbm_flattened_weights_s(int s, int half_width, int roots, int level, int max_level, int periodic,
                                     int k, double* out) {
  if (!out || s < 1 || s > 3 || half_width < 1 || half_width > 16 || roots < 1 || level < 0 ||
      max_level < level || max_level - level > 12 || level > 20)
    return MR_EINVAL;
  const long long N = (long long)roots << level;
  if (k < 0 || k >= N) return MR_EINVAL;
  const int W = half_width, gap = max_level - level, n = 1 << gap;
  // a window of the level around k: the true faces where k is within 2W + 2
  // cells of a non-periodic one, else an interior patch whose own faces lie
  // beyond every weight's reach (then periodic and interior cells agree)
  const int M = 4 * W + 5;
  int Nsim, ks;
  if (periodic || (k >= 2 * W + 2 && k <= N - 3 - 2 * W)) {
    Nsim = M;
    ks = 2 * W + 2;
  } else if (k < 2 * W + 2) {
    Nsim = (int)std::min<long long>(N, M);
    ks = k;
  } else {
    Nsim = (int)std::min<long long>(N, M);
    ks = (int)(k - (N - Nsim));
  }
  const bool lo_face = !periodic && k == 0, hi_face = !periodic && k == N - 1;
  for (int dl = -(W + 2); dl <= W + 2; ++dl) {
    const int i = ks + dl;
    double r0 = 0, r1 = 0, l0 = 0, l1 = 0;
    if (i >= 0 && i < Nsim) {
      std::vector<double> f(Nsim, 0.0);
      f[i] = 1.0;
      recon1d_s(f, Nsim, gap, s);
      if (!lo_face) r0 = f[(size_t)n * ks - 1];
      r1 = f[(size_t)n * (ks + 1) - 1];
      l0 = f[(size_t)n * ks];
      if (!hi_face) l1 = f[(size_t)n * (ks + 1)];
    }
    const double wp = r0 - r1, wm = l1 - l0;
    if (dl < -W || dl > W) {
      if (wp != 0.0 || wm != 0.0) return MR_EINVAL;  // the weights reach beyond the half-width
      continue;
    }
    out[dl + W] = wp;
    out[2 * W + 1 + dl + W] = wm;
  }
  return MR_OK;
}

mr_status mr_lbm_create(const mr_lbm_config* cfg, void* cuda_stream, mr_lbm_t* out) {
  if (!out) return MR_EINVAL;
  *out = nullptr;
  mr_status v = validate(cfg);
  if (v != MR_OK) return v;
  mr_lbm* h = new (std::nothrow) mr_lbm();
  if (!h) return MR_ENOMEM;
  Geo& g = h->g;
  memset(&g, 0, sizeof(g));
  g.scheme = cfg->scheme;
  if (!scheme_setup(g, cfg)) {
    delete h;
    return MR_EINVAL;
  }
  g.Jmin = cfg->min_level;
  g.J = cfg->max_level;
  for (int a = 0; a < 3; ++a) g.roots[a] = a < g.d ? std::max(1, cfg->roots[a]) : 1;
  // the root-prefixed codes of the finest level must fit the 32-bit code
  // arrays (the dense index space below, under 2^30, bounds them further)
  if (((uint64_t)g.roots[0] * g.roots[1] * g.roots[2] << (g.d * g.J)) > (1ull << 32)) {
    delete h;
    return MR_EINVAL;
  }
  uint64_t base = 0;
  for (int l = 0; l < MR_MAXL; ++l) {
    for (int a = 0; a < 3; ++a) g.n[l][a] = a < g.d ? (g.roots[a] << l) : 1;
    g.ncode[l] = (uint32_t)((uint64_t)g.n[l][0] * g.n[l][1] * g.n[l][2]);
  }
  for (int l = 0; l <= MR_MAXL; ++l) {
    g.base[l] = (uint32_t)base;
    if (l >= g.Jmin && l <= g.J) base += (g.ncode[l] + MR_DENSE_ALIGN - 1) / MR_DENSE_ALIGN * MR_DENSE_ALIGN;
  }
  if (base >= (1ull << 30)) {
    delete h;
    return MR_EINVAL;
  }
  for (int a = 0; a < 3; ++a) g.periodic[a] = a < g.d && cfg->bc[2 * a] == MR_BC_PERIODIC;
  for (int f = 0; f < 6; ++f) g.bc[f] = cfg->bc[f];
  g.lambda = cfg->lambda;
  g.inv_lambda = 1.0 / cfg->lambda;
  for (int i = 0; i < 16; ++i) g.s[i] = cfg->s[i];
  for (int i = 0; i < 8; ++i) g.phys[i] = cfg->phys[i];
  g.eps = cfg->eps;
  g.mu_bar = cfg->mu_bar;
  g.cross_sign = cfg->cross_sign == -1 ? -1 : 1;
  g.s_pred = cfg->pred_s ? cfg->pred_s : 1;
  g.form = cfg->precision;  // MR_FP64 .. MR_FP32_BF16STORE map onto MR_FORM_F64 .. MR_FORM_F32_BF16
  for (int p = 0; p < MR_MAXQ; ++p) g.off[p] = g.feq0[p] = g.bcv[p] = 0.0;
  g.diag = g.scheme == MR_D2Q9_NS;
  g.obstacle = cfg->obstacle;
  g.xlo[0] = cfg->xmin[0];
  g.xlo[1] = cfg->xmin[1];
  g.dxJ = (cfg->xmax[0] - cfg->xmin[0]) / g.n[g.J][0];
  for (int i = 0; i < 3; ++i) g.obs[i] = cfg->phys[3 + i];
  if (g.scheme == MR_D2Q9_NS) {
    // rest state (rho0, 0) of the obstacle; wall state (rho0, rho0 u0)
    const double rest[4] = {cfg->phys[0], 0.0, 0.0, 0.0};
    const double wall[4] = {cfg->phys[0], cfg->phys[0] * cfg->phys[1], cfg->phys[0] * cfg->phys[2], 0.0};
    double fw[MR_MAXQ];
    host_equilibrium(g, rest, g.feq0);
    host_equilibrium(g, wall, fw);
    for (int p = 0; p < g.Q; ++p) g.bcv[p] = fw[p] - fw[g.opp[p]];
  }
  long long nJ = g.ncode[g.J], nint = 0, nall = 0;
  for (int l = g.Jmin; l <= g.J; ++l) {
    nall += g.ncode[l];
    if (l < g.J) nint += g.ncode[l];
  }
  long long capL = cfg->leaf_capacity > 0 ? std::min<long long>(cfg->leaf_capacity, nJ) : nJ;
  g.cap[0] = (int)capL;
  g.cap[1] = (int)std::max<long long>(nint, 1);
  g.cap[2] = (int)nall;
  h->st = (cudaStream_t)cuda_stream;
  {
    const char* env = getenv("MR_LBM_GRAPHS");  // "0" launches every kernel directly
    h->use_graph = !(env && env[0] == '0');
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (h->nsm <= 0) h->nsm = 152;

  const size_t dense = g.base[g.J + 1];
  const size_t eb = mr_form_bytes(g.form);  // bytes per stored population value
  char *fs = nullptr, *fsc = nullptr;
  const size_t nch = dense / MR_DENSE_ALIGN;  // every level starts on a chunk boundary
  bool ok = dalloc(h, &h->cntbuf, 2) && dalloc(h, &h->flags, dense) && dalloc(h, &h->cls, dense) &&
            dalloc(h, &h->act, 2 * nch) && dalloc(h, &h->bcounts, 3 * (nch + 1)) && dalloc(h, &h->inidx, dense) &&
            dalloc(h, &h->vol, 1) && dalloc(h, &fs, eb * g.Q * g.cap[0]) && dalloc(h, &fsc, eb * g.Q * g.cap[0]);
  h->fstate = fs;
  h->fscratch = fsc;
  for (int mi = 0; mi < 2 && ok; ++mi) {
    MeshDev& M = h->mesh[mi];
    for (int c = 0; c < 3 && ok; ++c) ok = dalloc(h, &M.code[c], g.cap[c]) && dalloc(h, &M.lvl[c], g.cap[c]);
    char *ifp = nullptr, *gfp = nullptr;
    ok = ok && dalloc(h, &M.map, dense) && dalloc(h, &M.mact, nch) && dalloc(h, &ifp, eb * g.Q * g.cap[1]) &&
         dalloc(h, &gfp, eb * g.Q * g.cap[2]) && dalloc(h, &M.G, g.cap[1]) && dalloc(h, &M.src, g.cap[0]);
    M.IF = ifp;
    M.GF = gfp;
    if (ok) M.cnt = h->cntbuf + mi;
  }
  std::vector<double> W;
  build_tables(g, W);
  ok = ok && dalloc(h, &h->W, W.size()) && dalloc(h, &h->Wf, W.size());
  std::vector<float> Wf(W.begin(), W.end());
  if ((g.diag && g.s_pred == 1) || g.s_pred > 1) {  // critical-case details of the transport
    char* dp = nullptr;
    ok = ok && dalloc(h, &dp, ((size_t)1 << g.d) * g.Q * g.cap[1] * (g.form == MR_FORM_F64 ? 8 : 4));
    h->det = dp;
  }
  std::vector<double> Ws;
  if (g.s_pred > 1) {
    build_tables_w(g, Ws);
    ok = ok && dalloc(h, &h->Ws, Ws.size()) && dalloc(h, &h->Wsf, Ws.size());
  }
  std::vector<float> Wsf(Ws.begin(), Ws.end());
  int* dchunk = nullptr;
  ok = ok && dalloc(h, &h->dinst, 1) && dalloc(h, &dchunk, 2);
  if (!ok) {
    mr_lbm_destroy(h);
    return MR_ENOMEM;
  }
  if (!make_group(h->grp, {h}, h->dinst, dchunk, h->st, h->nsm) || !upload_desc(h)) {
    mr_lbm_destroy(h);
    return MR_ECUDA;
  }
  if (cfg->exact_collision) {
    h->grp.exact_nd = (long long)dense;
    if (!dalloc(h, &h->grp.exact, dense * g.Q)) {
      mr_lbm_destroy(h);
      return MR_ENOMEM;
    }
  }
  bool cok = cudaMemsetAsync(h->cntbuf, 0, 2 * sizeof(MeshCounts), h->st) == cudaSuccess &&
             cudaMemsetAsync(h->flags, 0, dense, h->st) == cudaSuccess &&
             cudaMemsetAsync(h->cls, 0, dense, h->st) == cudaSuccess &&
             cudaMemsetAsync(h->act, 0, 2 * nch, h->st) == cudaSuccess &&
             cudaMemsetAsync(h->mesh[0].mact, 0, nch, h->st) == cudaSuccess &&
             cudaMemsetAsync(h->mesh[1].mact, 0, nch, h->st) == cudaSuccess &&
             cudaMemsetAsync(h->inidx, 0xff, dense * sizeof(int32_t), h->st) == cudaSuccess &&
             cudaMemsetAsync(h->mesh[0].map, 0xff, dense * sizeof(int32_t), h->st) == cudaSuccess &&
             cudaMemsetAsync(h->mesh[1].map, 0xff, dense * sizeof(int32_t), h->st) == cudaSuccess &&
             cudaMemcpyAsync(h->Wf, Wf.data(), Wf.size() * sizeof(float), cudaMemcpyHostToDevice, h->st) ==
                 cudaSuccess &&
             cudaMemcpyAsync(h->W, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, h->st) ==
                 cudaSuccess &&
             (Ws.empty() || (cudaMemcpyAsync(h->Ws, Ws.data(), Ws.size() * sizeof(double), cudaMemcpyHostToDevice,
                                             h->st) == cudaSuccess &&
                             cudaMemcpyAsync(h->Wsf, Wsf.data(), Wsf.size() * sizeof(float),
                                             cudaMemcpyHostToDevice, h->st) == cudaSuccess)) &&
             cudaStreamSynchronize(h->st) == cudaSuccess;
  if (!cok) {
    mr_lbm_destroy(h);
    return MR_ECUDA;
  }
  *out = h;
  return MR_OK;
}

static void destroy_handle_impl(mr_lbm_t h);
static mr_status init_impl(mr_lbm_t h, const double* conserved, int on_device);

mr_status mr_lbm_destroy(mr_lbm_t h) {
  if (!h) return MR_OK;
  if (h->batch) return MR_ESTATE;  // owned by its batch
  destroy_handle_impl(h);
  return MR_OK;
}

mr_status mr_lbm_init(mr_lbm_t h, const double* conserved, int on_device) {
  if (!h || !conserved) return MR_EINVAL;
  if (h->sticky != MR_OK) return h->sticky;
  return init_impl(h, conserved, on_device);
}

static void destroy_handle_impl(mr_lbm_t h) {
  cudaStreamSynchronize(h->st);
  if (h->up_st) {
    cudaStreamSynchronize(h->up_st);
    cudaStreamDestroy(h->up_st);
    cudaEventDestroy(h->ev_prior);
    cudaEventDestroy(h->ev_up);
  }
  drop_graphs(*h);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  for (void* p : h->allocs) cudaFree(p);
  if (h->staging) cudaFree(h->staging);
  for (int i = 0; i < 2; ++i)
    if (h->dense[i]) cudaFree(h->dense[i]);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  delete h;
}

static mr_status init_impl(mr_lbm_t h, const double* conserved, int on_device) {
  const Geo& g = h->g;
  const size_t bytes = (size_t)g.ncons * g.ncode[g.J] * sizeof(double);
  const double* src = conserved;
  if (g.form == MR_FORM_F32_F16 || g.form == MR_FORM_F32_BF16) {
    // 16-bit storage keeps populations as offsets from the equilibrium of
    // the mean initial state
    std::vector<double> hc;
    const double* cp = conserved;
    if (on_device) {
      hc.resize(bytes / sizeof(double));
      if (!cuda_ok(h, cudaMemcpy(hc.data(), conserved, bytes, cudaMemcpyDeviceToHost))) return MR_ECUDA;
      cp = hc.data();
    }
    const long long N = g.ncode[g.J];
    double u[4] = {0, 0, 0, 0};
    for (int k = 0; k < g.ncons; ++k) {
      double s = 0;
      for (long long c = 0; c < N; ++c) s += cp[k * N + c];
      u[k] = s / (double)N;
    }
    host_equilibrium(h->g, u, h->g.off);
    if (!upload_desc(h)) return MR_ECUDA;
  }
  if (!on_device) {
    if (ensure_staging(h, bytes) != MR_OK) return h->sticky;
    if (!cuda_ok(h, cudaMemcpyAsync(h->staging, conserved, bytes, cudaMemcpyHostToDevice, h->st)))
      return MR_ECUDA;
    src = (const double*)h->staging;
  }
  MeshDev& B = h->mesh[h->cur];
  mr_launch_full_mesh(g, h->cls, h->act, h->st, grid_for(h));
  count_launch(h);
  run_build(*h, h->grp, h->cur);
  mr_launch_init_eq(g, B, src, h->fstate, h->st, grid_for(h));
  count_launch(h);
  if (check_launch(h) != MR_OK) return h->sticky;
  if (!on_device && !cuda_ok(h, cudaStreamSynchronize(h->st))) return MR_ECUDA;
  h->initialized = true;
  return MR_OK;
}

mr_status mr_lbm_step(mr_lbm_t h, int nsteps) {
  if (!h || nsteps < 0) return MR_EINVAL;
  if (h->sticky != MR_OK) return h->sticky;
  if (h->batch) return MR_ESTATE;  // the batch steps its instances
  if (!h->initialized) return fail(h, MR_ESTATE);
  queue_steps(*h, nsteps, [h]() { run_step(*h, h->grp, h->cur); });
  return check_launch(h);
}

mr_status mr_lbm_adapt(mr_lbm_t h) {
  if (!h) return MR_EINVAL;
  if (h->sticky != MR_OK) return h->sticky;
  if (h->batch) return MR_ESTATE;  // the batch steps its instances
  if (!h->initialized) return fail(h, MR_ESTATE);
  run_adapt(*h, h->grp, h->cur);
  std::swap(h->fstate, h->fscratch);
  if (!upload_desc(h)) return MR_ECUDA;  // the kernels read the buffers from the descriptor
  h->cur = 1 - h->cur;
  return check_launch(h);
}

mr_status mr_lbm_project(mr_lbm_t h, int level, double* out, int on_device) {
  if (!h || !out) return MR_EINVAL;
  if (h->sticky != MR_OK) return h->sticky;
  if (!h->initialized) return fail(h, MR_ESTATE);
  const Geo& g = h->g;
  if (level < g.Jmin || level > g.J) return MR_EINVAL;
  const size_t need = (size_t)g.ncons * g.ncode[g.J];
  if (h->dense_elems < need) {
    for (int i = 0; i < 2; ++i) {
      if (h->dense[i]) cudaFree(h->dense[i]);
      h->dense[i] = nullptr;
      if (cudaMalloc(&h->dense[i], need * sizeof(double)) != cudaSuccess) return fail(h, MR_ENOMEM);
    }
    h->dense_elems = need;
  }
  const MeshDev& A = h->mesh[h->cur];
  run_projection(*h, h->grp, h->cur);
  int pb = 0;
  for (int l = g.Jmin; l <= level; ++l) {
    mr_launch_project_dense(g, A, h->fstate, l, h->dense[pb], h->dense[1 - pb], h->st, grid_for(h));
    count_launch(h);
    pb = 1 - pb;
  }
  const double* res = h->dense[pb];
  const size_t bytes = (size_t)g.ncons * g.ncode[level] * sizeof(double);
  if (!cuda_ok(h, cudaMemcpyAsync(out, res, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  h->st)))
    return MR_ECUDA;
  if (check_launch(h) != MR_OK) return h->sticky;
  if (!on_device) {
    MeshCounts hc[2];
    return read_counts(h, hc);
  }
  return MR_OK;
}

mr_status mr_lbm_get_leaves(mr_lbm_t h, long long* n_inout, unsigned long long* keys, signed char* levels,
                            double* f, int on_device) {
  if (!h || !n_inout) return MR_EINVAL;
  if (h->sticky != MR_OK) return h->sticky;
  if (!h->initialized) return fail(h, MR_ESTATE);
  MeshCounts hc[2];
  mr_status s = read_counts(h, hc);
  if (s != MR_OK) return s;
  const long long n = hc[h->cur].total[MR_CLS_LEAF];
  if (!keys && !levels && !f) {
    *n_inout = n;
    return MR_OK;
  }
  if (*n_inout < n) return MR_EINVAL;
  const Geo& g = h->g;
  const MeshDev& A = h->mesh[h->cur];
  if (on_device) {
    mr_launch_leaves_out(g, A, h->fstate, n, keys, levels, f, h->st, grid_for(h));
    count_launch(h);
  } else {
    const size_t bk = n * sizeof(unsigned long long), bl = (n * sizeof(signed char) + 255) / 256 * 256,
                 bf = (size_t)g.Q * n * sizeof(double);
    if (ensure_staging(h, bk + bl + bf) != MR_OK) return h->sticky;
    char* sp = (char*)h->staging;
    mr_launch_leaves_out(g, A, h->fstate, n, (unsigned long long*)sp, (signed char*)(sp + bk),
                         (double*)(sp + bk + bl), h->st, grid_for(h));
    count_launch(h);
    if (keys && !cuda_ok(h, cudaMemcpyAsync(keys, sp, bk, cudaMemcpyDeviceToHost, h->st))) return MR_ECUDA;
    if (levels && !cuda_ok(h, cudaMemcpyAsync(levels, sp + bk, n, cudaMemcpyDeviceToHost, h->st)))
      return MR_ECUDA;
    if (f && !cuda_ok(h, cudaMemcpyAsync(f, sp + bk + bl, bf, cudaMemcpyDeviceToHost, h->st))) return MR_ECUDA;
    if (!cuda_ok(h, cudaStreamSynchronize(h->st))) return MR_ECUDA;
  }
  *n_inout = n;
  return check_launch(h);
}

mr_status mr_lbm_set_leaves(mr_lbm_t h, long long n, const unsigned long long* keys, const signed char* levels,
                            const double* f, int on_device) {
  if (!h || n <= 0 || !keys || !levels || !f) return MR_EINVAL;
  if (h->sticky != MR_OK) return h->sticky;
  const Geo& g = h->g;
  if (n > g.cap[0]) return fail(h, MR_ECAPACITY);
  if (!h->initialized && (g.form == MR_FORM_F32_F16 || g.form == MR_FORM_F32_BF16)) {
    // first state of the handle: 16-bit storage offsets = mean populations
    std::vector<double> hf;
    const double* fp = f;
    if (on_device) {
      hf.resize((size_t)g.Q * n);
      if (!cuda_ok(h, cudaMemcpy(hf.data(), f, hf.size() * sizeof(double), cudaMemcpyDeviceToHost)))
        return MR_ECUDA;
      fp = hf.data();
    }
    for (int p = 0; p < g.Q; ++p) {
      double s = 0;
      for (long long i = 0; i < n; ++i) s += fp[(size_t)p * n + i];
      h->g.off[p] = s / (double)n;
    }
    if (!upload_desc(h)) return MR_ECUDA;
  }
  const unsigned long long* dk = keys;
  const signed char* dl = levels;
  const double* df = f;
  bool up = false;  // populations in flight on up_st
  // error returns: the caller's host buffers are free on return, so wait for
  // the population upload to finish (after which nothing reads them)
  auto release = [&]() {
    if (up) cudaStreamSynchronize(h->up_st);
    up = false;
  };
  if (!on_device) {
    const size_t bk = n * sizeof(unsigned long long), bl = (n + 255) / 256 * 256, bf = (size_t)g.Q * n * sizeof(double);
    if (ensure_staging(h, bk + bl + bf) != MR_OK) return h->sticky;
    if (!h->up_st && (!cuda_ok(h, cudaStreamCreateWithFlags(&h->up_st, cudaStreamNonBlocking)) ||
                      !cuda_ok(h, cudaEventCreateWithFlags(&h->ev_prior, cudaEventDisableTiming)) ||
                      !cuda_ok(h, cudaEventCreateWithFlags(&h->ev_up, cudaEventDisableTiming))))
      return MR_ECUDA;
    char* sp = (char*)h->staging;
    // the populations (most of the bytes) go up on the second stream, after
    // the handle stream's earlier work (which may still read the staging
    // buffer), while the keys are checked and the mesh is built
    if (!cuda_ok(h, cudaEventRecord(h->ev_prior, h->st)) ||
        !cuda_ok(h, cudaStreamWaitEvent(h->up_st, h->ev_prior, 0)))
      return MR_ECUDA;
    if (!cuda_ok(h, cudaMemcpyAsync(sp + bk + bl, f, bf, cudaMemcpyHostToDevice, h->up_st))) return MR_ECUDA;
    up = true;
    if (!cuda_ok(h, cudaEventRecord(h->ev_up, h->up_st))) {
      release();
      return MR_ECUDA;
    }
    if (!cuda_ok(h, cudaMemcpyAsync(sp, keys, bk, cudaMemcpyHostToDevice, h->st)) ||
        !cuda_ok(h, cudaMemcpyAsync(sp + bk, levels, n, cudaMemcpyHostToDevice, h->st))) {
      release();
      return MR_ECUDA;
    }
    dk = (const unsigned long long*)sp;
    dl = (const signed char*)(sp + bk);
    df = (const double*)(sp + bk + bl);
  }
  // the success path orders the handle's stream after the upload
  auto join = [&]() {
    if (up) cudaStreamWaitEvent(h->st, h->ev_up, 0);
    up = false;
  };
  MeshDev& B = h->mesh[h->cur];
  if (!cuda_ok(h, cudaMemsetAsync(h->vol, 0, sizeof(unsigned long long), h->st))) {
    release();
    return MR_ECUDA;
  }
  mr_launch_leaves_in(g, n, dk, dl, h->inidx, h->cls, h->act, B.cnt, h->vol, h->st, grid_for(h));
  mr_launch_leaves_check(g, h->cls, B.cnt, h->st, grid_for(h));
  count_launch(h, 2);
  unsigned long long vol = 0;
  if (!cuda_ok(h, cudaMemcpyAsync(&vol, h->vol, sizeof(vol), cudaMemcpyDeviceToHost, h->st))) {
    release();
    return MR_ECUDA;
  }
  MeshCounts hc[2];
  mr_status s = read_counts(h, hc);
  if (s != MR_OK) {
    release();
    return s;
  }
  unsigned long long full = g.ncode[g.J];
  if (vol != full) {
    release();
    return fail(h, MR_EINVAL);
  }
  run_build(*h, h->grp, h->cur);
  join();
  mr_launch_gather_input(g, B, h->inidx, n, df, h->fstate, h->st, grid_for(h));
  count_launch(h);
  // reset the input index map for the next call
  if (!cuda_ok(h, cudaMemsetAsync(h->inidx, 0xff, (size_t)g.base[g.J + 1] * sizeof(int32_t), h->st)))
    return MR_ECUDA;
  if (check_launch(h) != MR_OK) return h->sticky;
  // the caller's buffers are free once the upload is done; errors of the
  // build and the gather come back at the next synchronising call
  if (!on_device && !cuda_ok(h, cudaEventSynchronize(h->ev_up))) return MR_ECUDA;
  h->initialized = true;
  return MR_OK;
}

mr_status mr_lbm_stats(mr_lbm_t h, long long* leaves_per_level, double* mesh_or, double* mem_or) {
  if (!h) return MR_EINVAL;
  if (h->sticky != MR_OK) return h->sticky;
  if (!h->initialized) return fail(h, MR_ESTATE);
  MeshCounts hc[2];
  mr_status s = read_counts(h, hc);
  if (s != MR_OK) return s;
  const MeshCounts& c = hc[h->cur];
  const Geo& g = h->g;
  if (leaves_per_level)
    for (int l = 0; l <= g.J; ++l)
      leaves_per_level[l] = l < g.Jmin ? 0 : c.off[MR_CLS_LEAF][l + 1] - c.off[MR_CLS_LEAF][l];
  double all = 0;
  for (int l = g.Jmin; l <= g.J; ++l) all += g.ncode[l];
  if (mesh_or) *mesh_or = (double)c.total[MR_CLS_LEAF] / (double)g.ncode[g.J];
  if (mem_or) *mem_or = (double)(c.total[MR_CLS_LEAF] + c.total[MR_CLS_INT]) / all;
  return MR_OK;
}

mr_status mr_lbm_counters(mr_lbm_t h, long long* leaf_updates, long long* steps) {
  if (!h) return MR_EINVAL;
  if (h->sticky != MR_OK) return h->sticky;
  MeshCounts hc[2];
  mr_status s = read_counts(h, hc);
  if (s != MR_OK) return s;
  if (leaf_updates) *leaf_updates = hc[0].leaf_updates + hc[1].leaf_updates;
  if (steps) *steps = hc[0].steps + hc[1].steps;
  return MR_OK;
}

long long mr_lbm_launch_count(mr_lbm_t h) { return h ? h->launches : 0; }

mr_status mr_lbm_profile_enable(mr_lbm_t h, int on) {
  if (!h || on < 0 || on > 6) return MR_EINVAL;
  if (!cuda_ok(h, cudaStreamSynchronize(h->st))) return MR_ECUDA;
  h->prof_group = on;
  h->ev_used = 0;
  return MR_OK;
}

mr_status mr_lbm_profile_read(mr_lbm_t h, double* total_ms, long long* launches) {
  if (!h) return MR_EINVAL;
  if (!cuda_ok(h, cudaStreamSynchronize(h->st))) return MR_ECUDA;
  const double tot = profile_total(*h, launches);
  if (tot < 0) return fail(h, MR_ECUDA);
  if (total_ms) *total_ms = tot;
  return MR_OK;
}

mr_status mr_lbm_synchronize(mr_lbm_t h) {
  if (!h) return MR_EINVAL;
  if (h->sticky != MR_OK) return h->sticky;
  MeshCounts hc[2];
  return read_counts(h, hc);
}

}  // extern "C"

// ----------------------------------------------------------------- adjoint
namespace {

// Device memory owned by one adjoint run, released on every return path.
struct AdjArena {
  std::vector<void*> blocks;
  ~AdjArena() {
    for (void* p : blocks) cudaFree(p);
  }
  template <class T>
  T* get(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, (count ? count : 1) * sizeof(T)) != cudaSuccess) return nullptr;
    blocks.push_back(p);
    return (T*)p;
  }
};

// Structure of one mesh (what the adjoint kernels read), copied aside.
struct MeshSnap {
  MeshDev m;
};

bool snap_alloc(AdjArena& ar, const Geo& g, MeshSnap& s) {
  const size_t dense = g.base[g.J + 1];
  memset(&s.m, 0, sizeof(s.m));
  bool ok = (s.m.map = ar.get<int32_t>(dense)) && (s.m.src = ar.get<int32_t>(g.cap[0])) &&
            (s.m.cnt = ar.get<MeshCounts>(1));
  for (int c = 0; c < 3 && ok; ++c) ok = (s.m.code[c] = ar.get<uint32_t>(g.cap[c])) && (s.m.lvl[c] = ar.get<uint8_t>(g.cap[c]));
  return ok;
}

bool snap_copy(const Geo& g, const MeshDev& from, MeshSnap& s, cudaStream_t st) {
  const size_t dense = g.base[g.J + 1];
  bool ok = cudaMemcpyAsync(s.m.map, from.map, dense * sizeof(int32_t), cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(s.m.src, from.src, g.cap[0] * sizeof(int32_t), cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(s.m.cnt, from.cnt, sizeof(MeshCounts), cudaMemcpyDeviceToDevice, st) == cudaSuccess;
  for (int c = 0; c < 3 && ok; ++c)
    ok = cudaMemcpyAsync(s.m.code[c], from.code[c], g.cap[c] * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) ==
             cudaSuccess &&
         cudaMemcpyAsync(s.m.lvl[c], from.lvl[c], g.cap[c], cudaMemcpyDeviceToDevice, st) == cudaSuccess;
  return ok;
}

// A saved state: the leaves of the current mesh (keys, levels, FP64 values).
struct Checkpoint {
  unsigned long long* keys = nullptr;
  signed char* levels = nullptr;
  double* f = nullptr;
  long long n = 0;
};

mr_status save_state(mr_lbm* h, AdjArena& ar, Checkpoint& c) {
  MeshCounts hc[2];
  mr_status s = read_counts(h, hc);
  if (s != MR_OK) return s;
  c.n = hc[h->cur].total[MR_CLS_LEAF];
  if (!c.keys) {
    c.keys = ar.get<unsigned long long>(h->g.cap[0]);
    c.levels = ar.get<signed char>(h->g.cap[0]);
    c.f = ar.get<double>((size_t)h->g.Q * h->g.cap[0]);
    if (!c.keys || !c.levels || !c.f) return fail(h, MR_ENOMEM);
  }
  mr_launch_leaves_out(h->g, h->mesh[h->cur], h->fstate, c.n, c.keys, c.levels, c.f, h->st, grid_for(h));
  h->launches += 1;
  return check_launch(h);
}

}  // namespace

extern "C" {

mr_status mr_lbm_adjoint(mr_lbm_t h, const double* conserved0, int on_device, int nsteps, int checkpoint_every,
                         int functional, double* J_out, double* grad_conserved0, double* grad_s) {
  if (!h || !conserved0 || nsteps < 1 || checkpoint_every < 1) return MR_EINVAL;
  if (functional != MR_FUNCTIONAL_KE_SUM && functional != MR_FUNCTIONAL_KE_FINAL) return MR_EINVAL;
  if (h->sticky != MR_OK) return h->sticky;
  if (h->batch) return MR_ESTATE;
  const Geo& g = h->g;
  if (g.form != MR_FORM_F64 || h->grp.exact || g.d == 3 || g.s_pred > 1) return MR_EINVAL;  // 1D and 2D, the leaf collision
  AdjArena ar;
  const size_t NJ = g.ncode[g.J], ncb = (size_t)g.ncons * NJ;
  // the initial field, kept on the device for the equilibrium's adjoint
  double* cons = ar.get<double>(ncb);
  double* dJ = ar.get<double>(1);
  double* ds = ar.get<double>(16);
  if (!cons || !dJ || !ds) return fail(h, MR_ENOMEM);
  if (!cuda_ok(h, cudaMemcpyAsync(cons, conserved0, ncb * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st)) ||
      !cuda_ok(h, cudaMemsetAsync(dJ, 0, sizeof(double), h->st)) ||
      !cuda_ok(h, cudaMemsetAsync(ds, 0, 16 * sizeof(double), h->st)))
    return MR_ECUDA;
  mr_status s = mr_lbm_init(h, cons, 1);
  if (s != MR_OK) return s;
  const int K = checkpoint_every, nseg = (nsteps + K - 1) / K;
  const double vol_J = g.d == 1 ? g.dxJ : g.d == 2 ? g.dxJ * g.dxJ : g.dxJ * g.dxJ * g.dxJ;
  const int grid = grid_for(h, 4);
  std::vector<Checkpoint> cps(nseg + 1);
  // forward pass: the functional and a checkpoint every K steps
  for (int n = 0; n < nsteps; ++n) {
    if (n % K == 0 && (s = save_state(h, ar, cps[n / K])) != MR_OK) return s;
    queue_steps(*h, 1, [h]() { run_step(*h, h->grp, h->cur); });
    if (functional == MR_FUNCTIONAL_KE_SUM || n == nsteps - 1) {
      mr_kinetic_energy(g, h->mesh[h->cur], (const double*)h->fstate, vol_J, dJ, h->st, grid);
      h->launches += 1;
    }
  }
  if ((s = check_launch(h)) != MR_OK) return s;
  if (J_out && !cuda_ok(h, cudaMemcpyAsync(J_out, dJ, sizeof(double), cudaMemcpyDeviceToHost, h->st))) return MR_ECUDA;
  if (!grad_conserved0 && !grad_s) return mr_lbm_synchronize(h);
  if ((s = save_state(h, ar, cps[nseg])) != MR_OK) return s;  // the final state, restored at the end

  // backward pass, one segment at a time: replay the segment from its
  // checkpoint recording meshes and pre-collision states, then sweep back
  const size_t QL = (size_t)g.Q * g.cap[0];
  double* lam = ar.get<double>(QL);
  double* aLB = ar.get<double>(QL);
  double* aIB = ar.get<double>((size_t)g.Q * g.cap[1]);
  double* aGB = ar.get<double>((size_t)g.Q * g.cap[2]);
  double* aIA = ar.get<double>((size_t)g.Q * g.cap[1]);
  double* aLA = ar.get<double>(QL);
  std::vector<MeshSnap> tape(K + 1);
  std::vector<double*> z(K);
  bool ok = lam && aLB && aIB && aGB && aIA && aLA;
  for (int j = 0; j <= K && ok; ++j) ok = snap_alloc(ar, g, tape[j]) && (j == K || (z[j] = ar.get<double>(QL)));
  if (!ok) return fail(h, MR_ENOMEM);
  if (!cuda_ok(h, cudaMemsetAsync(lam, 0, QL * sizeof(double), h->st))) return MR_ECUDA;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int n0 = sg * K, n1 = std::min(nsteps, n0 + K);
    const Checkpoint& c = cps[sg];
    if ((s = mr_lbm_set_leaves(h, c.n, c.keys, c.levels, c.f, 1)) != MR_OK) return s;
    if (!snap_copy(g, h->mesh[h->cur], tape[0], h->st)) return fail(h, MR_ECUDA);
    for (int n = n0; n < n1; ++n) {
      const int j = n - n0;
      run_adapt(*h, h->grp, h->cur);
      if (g.scheme == MR_D2Q9_NS) {  // the transport's critical-case details
        mr_launch_edge_details(h->grp, 1 - h->cur, h->st);
        h->launches += 1;
      }
      mr_launch_stream_collide(h->grp, 1 - h->cur, 1, 0, h->st);  // stored state <- transport only
      if (!cuda_ok(h, cudaMemcpyAsync(z[j], h->fstate, QL * sizeof(double), cudaMemcpyDeviceToDevice, h->st)) ||
          !cuda_ok(h, cudaMemcpyAsync(h->fscratch, h->fstate, QL * sizeof(double), cudaMemcpyDeviceToDevice, h->st)))
        return MR_ECUDA;
      mr_launch_stream_collide(h->grp, 1 - h->cur, 0, 1, h->st);  // collision (and obstacle) of it
      h->launches += 2;
      h->cur = 1 - h->cur;
      if (!snap_copy(g, h->mesh[h->cur], tape[j + 1], h->st)) return fail(h, MR_ECUDA);
    }
    for (int n = n1 - 1; n >= n0; --n) {
      const int j = n - n0;
      const MeshDev& A = tape[j].m;
      const MeshDev& B = tape[j + 1].m;
      const int src = functional == MR_FUNCTIONAL_KE_SUM || n == nsteps - 1;
      mr_adj_collide(g, B, z[j], lam, ds, src, vol_J, h->st, grid);
      bool zok = cudaMemsetAsync(aLB, 0, QL * sizeof(double), h->st) == cudaSuccess &&
                 cudaMemsetAsync(aIB, 0, (size_t)g.Q * g.cap[1] * sizeof(double), h->st) == cudaSuccess &&
                 cudaMemsetAsync(aGB, 0, (size_t)g.Q * g.cap[2] * sizeof(double), h->st) == cudaSuccess &&
                 cudaMemsetAsync(aLA, 0, QL * sizeof(double), h->st) == cudaSuccess &&
                 cudaMemsetAsync(aIA, 0, (size_t)g.Q * g.cap[1] * sizeof(double), h->st) == cudaSuccess;
      if (!cuda_ok(h, zok ? cudaSuccess : cudaErrorUnknown)) return MR_ECUDA;
      mr_adj_transport(g, B, h->W, lam, aLB, aIB, aGB, h->st, grid);
      for (int l = g.J; l > g.Jmin; --l) mr_adj_predict(g, B, l, aLB, aIB, aGB, h->st, grid);
      mr_adj_transfer(g, A, B, aLB, aIB, aLA, aIA, h->st, grid);
      for (int l = g.Jmin; l < g.J; ++l) mr_adj_project(g, A, l, aLA, aIA, h->st, grid);
      h->launches += 3 + 2 * (g.J - g.Jmin);
      std::swap(lam, aLA);
    }
    if ((s = check_launch(h)) != MR_OK) return s;
  }
  // lam: adjoint of the initial populations on the full finest mesh
  double* grad = ar.get<double>(ncb);
  if (!grad) return fail(h, MR_ENOMEM);
  mr_adj_init(g, tape[0].m, cons, lam, grad, h->st, grid);
  h->launches += 1;
  if (grad_conserved0 &&
      !cuda_ok(h, cudaMemcpyAsync(grad_conserved0, grad, ncb * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st)))
    return MR_ECUDA;
  if (grad_s && !cuda_ok(h, cudaMemcpyAsync(grad_s, ds, 16 * sizeof(double), cudaMemcpyDeviceToHost, h->st)))
    return MR_ECUDA;
  // device errors of the tape meshes (the adjoint kernels flag there)
  std::vector<MeshCounts> tc(K + 1);
  for (int j = 0; j <= K; ++j)
    if (!cuda_ok(h, cudaMemcpyAsync(&tc[j], tape[j].m.cnt, sizeof(MeshCounts), cudaMemcpyDeviceToHost, h->st)))
      return MR_ECUDA;
  if (!cuda_ok(h, cudaStreamSynchronize(h->st))) return MR_ECUDA;
  for (int j = 0; j <= K; ++j)
    if (tc[j].err & MR_DERR_INTERNAL) return fail(h, MR_EINTERNAL);
  const Checkpoint& last = cps[nseg];
  return mr_lbm_set_leaves(h, last.n, last.keys, last.levels, last.f, 1);
}

}  // extern "C"

// ----------------------------------------------------------------- batches
struct mr_lbm_batch : Exec {
  std::vector<mr_lbm*> inst;  // in the caller's order
  struct Part {               // instances of one scheme and form, contiguous in descs
    Group G;
    int* chunk_pre = nullptr;
    cudaStream_t side = nullptr;  // branch stream of the parts after the first
    cudaEvent_t done = nullptr;
  };
  std::vector<Part> parts;
  InstDev* descs = nullptr;
  cudaEvent_t fork = nullptr;
  mr_status sticky = MR_OK;
};

namespace {

// One step of every instance: one chain of launches per part, the parts
// after the first on branch streams forked from and joined to b->st.
void run_batch_step(mr_lbm_batch* b) {
  const int cur = b->cur;
  cudaStream_t main = b->st;
  const size_t np = b->parts.size();
  if (np > 1) {
    cudaEventRecord(b->fork, main);
    for (size_t p = 1; p < np; ++p) cudaStreamWaitEvent(b->parts[p].side, b->fork, 0);
  }
  for (size_t p = 0; p < np; ++p) {
    b->st = p == 0 ? main : b->parts[p].side;
    run_step(*b, b->parts[p].G, cur);
  }
  b->st = main;
  for (size_t p = 1; p < np; ++p) {
    cudaEventRecord(b->parts[p].done, b->parts[p].side);
    cudaStreamWaitEvent(main, b->parts[p].done, 0);
  }
}

void free_batch(mr_lbm_batch* b) {
  if (b->st) cudaStreamSynchronize(b->st);
  drop_graphs(*b);
  if (b->cap_st) cudaStreamDestroy(b->cap_st);
  for (auto& p : b->parts) {
    if (p.side) cudaStreamDestroy(p.side);
    if (p.done) cudaEventDestroy(p.done);
    if (p.chunk_pre) cudaFree(p.chunk_pre);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  for (mr_lbm* h : b->inst)
    if (h) {
      h->batch = nullptr;
      destroy_handle_impl(h);
    }
  if (b->descs) cudaFree(b->descs);
  for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
  delete b;
}

// ---- launch schedules: the autotuner's cache
// A batch's signature names each part by half-width, scheme, form, size and
// the power of two of its mean finest-cell count; the cache maps it to the
// parts' schedules (MR_NPH blocks-per-SM values each).  It lives in the
// process and, when MR_LBM_TUNE_CACHE names a file, in that file (one line
// per tuning, the last line of a signature wins).
std::mutex g_tune_mutex;
std::map<std::string, std::vector<int>> g_tune_cache;
bool g_tune_file_read = false;

std::string batch_signature(const mr_lbm_batch* b) {
  std::string sig;
  for (const auto& p : b->parts) {
    const long long avg = std::max<long long>(1, p.G.capL / std::max(1, p.G.n));
    int band = 0;
    while ((1ll << (band + 1)) <= avg) ++band;
    char buf[96];
    snprintf(buf, sizeof buf, "%d.%d.%d.%d.%d/", p.G.s, p.G.scheme, p.G.form, p.G.n, band);
    sig += buf;
  }
  return sig;
}

void tune_cache_read_file() {  // under g_tune_mutex
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char* path = getenv("MR_LBM_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* fp = fopen(path, "r");
  if (!fp) return;
  char line[4096];
  while (fgets(line, sizeof line, fp)) {
    char* save = nullptr;
    char* tok = strtok_r(line, " \t\n", &save);
    if (!tok) continue;
    std::string sig = tok;
    std::vector<int> v;
    while ((tok = strtok_r(nullptr, " \t\n", &save))) v.push_back(atoi(tok));
    if (!v.empty()) g_tune_cache[sig] = v;
  }
  fclose(fp);
}

// Schedules of a batch's parts from the cache, if it holds its signature.
void apply_cached_schedule(mr_lbm_batch* b) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_cache_read_file();
  auto it = g_tune_cache.find(batch_signature(b));
  if (it == g_tune_cache.end() || it->second.size() != b->parts.size() * MR_NPH) return;
  for (size_t p = 0; p < b->parts.size(); ++p)
    for (int ph = 0; ph < MR_NPH; ++ph) {
      const int v = it->second[p * MR_NPH + ph];
      if (v >= 1 && v <= 64) b->parts[p].G.bps[ph] = v;
    }
}

void store_schedule(const mr_lbm_batch* b) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  tune_cache_read_file();
  std::vector<int> v;
  for (const auto& p : b->parts) v.insert(v.end(), p.G.bps, p.G.bps + MR_NPH);
  const std::string sig = batch_signature(b);
  g_tune_cache[sig] = v;
  const char* path = getenv("MR_LBM_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* fp = fopen(path, "a");
  if (!fp) return;
  fprintf(fp, "%s", sig.c_str());
  for (int x : v) fprintf(fp, " %d", x);
  fprintf(fp, "\n");
  fclose(fp);
}

}  // namespace

extern "C" {

mr_status mr_lbm_batch_create(const mr_lbm_config* cfgs, int n, void* cuda_stream, mr_lbm_batch_t* out) {
  if (!out) return MR_EINVAL;
  *out = nullptr;
  if (!cfgs || n <= 0) return MR_EINVAL;
  for (int i = 0; i < n; ++i)
    if (cfgs[i].exact_collision) return MR_EINVAL;  // single solvers only
  mr_lbm_batch* b = new (std::nothrow) mr_lbm_batch();
  if (!b) return MR_ENOMEM;
  b->st = (cudaStream_t)cuda_stream;
  b->inst.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    const mr_status s = mr_lbm_create(&cfgs[i], cuda_stream, &b->inst[i]);
    if (s != MR_OK) {
      free_batch(b);
      return s;
    }
  }
  b->nsm = b->inst[0]->nsm;
  // parts: instances of one scheme and storage form, at most MR_MAXB each
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto key = [&](int i) { return (b->inst[i]->g.s_pred * 16 + b->inst[i]->g.scheme) * 16 + b->inst[i]->g.form; };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key(x) < key(y); });
  if (cudaMalloc(&b->descs, sizeof(InstDev) * n) != cudaSuccess) {
    free_batch(b);
    return MR_ENOMEM;
  }
  bool ok = true;
  for (int s = 0; s < n && ok;) {
    int e = s + 1;
    while (e < n && e - s < MR_MAXB && key(order[e]) == key(order[s])) ++e;
    mr_lbm_batch::Part part;
    std::vector<const mr_lbm*> members;
    for (int k = s; k < e; ++k) {
      mr_lbm* h = b->inst[order[k]];
      h->batch = b;
      h->dinst = b->descs + k;
      h->grp.dev = h->dinst;
      ok = ok && upload_desc(h);
      members.push_back(h);
    }
    ok = ok && cudaMalloc(&part.chunk_pre, sizeof(int) * (e - s + 1)) == cudaSuccess &&
         make_group(part.G, members, b->descs + s, part.chunk_pre, b->st, b->nsm);
    if (ok && !b->parts.empty())
      ok = cudaStreamCreateWithFlags(&part.side, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&part.done, cudaEventDisableTiming) == cudaSuccess;
    b->parts.push_back(part);
    s = e;
  }
  ok = ok && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
       cudaStreamSynchronize(b->st) == cudaSuccess;
  if (!ok) {
    free_batch(b);
    return MR_ECUDA;
  }
  apply_cached_schedule(b);
  *out = b;
  return MR_OK;
}

mr_status mr_lbm_batch_instance(mr_lbm_batch_t b, int i, mr_lbm_t* out) {
  if (!b || !out || i < 0 || i >= (int)b->inst.size()) return MR_EINVAL;
  *out = b->inst[i];
  return MR_OK;
}

mr_status mr_lbm_batch_step(mr_lbm_batch_t b, int nsteps) {
  if (!b || nsteps < 0) return MR_EINVAL;
  if (b->sticky != MR_OK) return b->sticky;
  for (mr_lbm* h : b->inst) {
    if (h->sticky != MR_OK) return h->sticky;
    if (!h->initialized || h->cur != b->cur) return MR_ESTATE;
  }
  queue_steps(*b, nsteps, [b]() { run_batch_step(b); });
  for (mr_lbm* h : b->inst) h->cur = b->cur;
  if (cudaGetLastError() != cudaSuccess) b->sticky = MR_ECUDA;
  return b->sticky;
}

mr_status mr_lbm_batch_synchronize(mr_lbm_batch_t b) {
  if (!b) return MR_EINVAL;
  if (b->sticky != MR_OK) return b->sticky;
  mr_status first = MR_OK;
  for (mr_lbm* h : b->inst) {
    const mr_status s = mr_lbm_synchronize(h);
    if (first == MR_OK) first = s;
  }
  return first;
}

mr_status mr_lbm_batch_counters(mr_lbm_batch_t b, long long* leaf_updates, long long* steps) {
  if (!b) return MR_EINVAL;
  long long lu = 0, st = 0;
  for (mr_lbm* h : b->inst) {
    long long a = 0, c = 0;
    const mr_status s = mr_lbm_counters(h, &a, &c);
    if (s != MR_OK) return s;
    lu += a;
    st = std::max(st, c);
  }
  if (leaf_updates) *leaf_updates = lu;
  if (steps) *steps = st;
  return MR_OK;
}

long long mr_lbm_batch_launch_count(mr_lbm_batch_t b) { return b ? b->launches : 0; }

mr_status mr_lbm_batch_profile_enable(mr_lbm_batch_t b, int on) {
  if (!b || on < 0 || on > 6) return MR_EINVAL;
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return MR_ECUDA;
  b->prof_group = on;
  b->ev_used = 0;
  return MR_OK;
}

mr_status mr_lbm_batch_profile_read(mr_lbm_batch_t b, double* total_ms, long long* launches) {
  if (!b) return MR_EINVAL;
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return MR_ECUDA;
  const double tot = profile_total(*b, launches);
  if (tot < 0) return MR_ECUDA;
  if (total_ms) *total_ms = tot;
  return MR_OK;
}

mr_status mr_lbm_batch_parts(mr_lbm_batch_t b, int* nparts) {
  if (!b || !nparts) return MR_EINVAL;
  *nparts = (int)b->parts.size();
  return MR_OK;
}

mr_status mr_lbm_batch_get_schedule(mr_lbm_batch_t b, int part, int* bps) {
  if (!b || !bps || part < 0 || part >= (int)b->parts.size()) return MR_EINVAL;
  for (int ph = 0; ph < MR_NPH; ++ph) bps[ph] = b->parts[part].G.bps[ph];
  return MR_OK;
}

mr_status mr_lbm_batch_set_schedule(mr_lbm_batch_t b, int part, const int* bps) {
  if (!b || !bps || part < 0 || part >= (int)b->parts.size()) return MR_EINVAL;
  for (int ph = 0; ph < MR_NPH; ++ph)
    if (bps[ph] < 1 || bps[ph] > 64) return MR_EINVAL;
  if (b->st && cudaStreamSynchronize(b->st) != cudaSuccess) return MR_ECUDA;
  for (int ph = 0; ph < MR_NPH; ++ph) b->parts[part].G.bps[ph] = bps[ph];
  drop_graphs(*b);  // the captured steps carry the old grids
  return MR_OK;
}

mr_status mr_lbm_batch_autotune(mr_lbm_batch_t b, int trial_steps, double* ms_fixed, double* ms_tuned) {
  if (!b || trial_steps < 1 || trial_steps > 1000) return MR_EINVAL;
  if (b->sticky != MR_OK) return b->sticky;
  for (mr_lbm* h : b->inst) {
    if (h->sticky != MR_OK) return h->sticky;
    if (!h->initialized || h->cur != b->cur) return MR_ESTATE;
  }
  const size_t ni = b->inst.size();
  // snapshot of every instance: leaves, counters and launch counts
  struct Snap {
    long long n = 0;
    unsigned long long* k = nullptr;
    signed char* l = nullptr;
    double* f = nullptr;
    MeshCounts cnt[2];
    long long launches = 0;
  };
  std::vector<Snap> snap(ni);
  const long long launches0 = b->launches;
  mr_status st = MR_OK;
  auto release = [&]() {
    for (Snap& s : snap) {
      if (s.k) cudaFree(s.k);
      if (s.l) cudaFree(s.l);
      if (s.f) cudaFree(s.f);
    }
  };
  for (size_t i = 0; i < ni && st == MR_OK; ++i) {
    mr_lbm* h = b->inst[i];
    Snap& s = snap[i];
    st = mr_lbm_get_leaves(h, &s.n, nullptr, nullptr, nullptr, 1);
    if (st != MR_OK) break;
    if (cudaMalloc(&s.k, s.n * sizeof(unsigned long long)) != cudaSuccess || cudaMalloc(&s.l, s.n) != cudaSuccess ||
        cudaMalloc(&s.f, (size_t)h->g.Q * s.n * sizeof(double)) != cudaSuccess) {
      st = MR_ENOMEM;
      break;
    }
    long long n = s.n;
    st = mr_lbm_get_leaves(h, &n, s.k, s.l, s.f, 1);
    if (st == MR_OK && cudaMemcpy(s.cnt, h->cntbuf, 2 * sizeof(MeshCounts), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = MR_ECUDA;
    s.launches = h->launches;
  }
  if (st != MR_OK) {
    release();
    return st;
  }
  auto restore = [&]() -> mr_status {
    for (size_t i = 0; i < ni; ++i) {
      const mr_status r = mr_lbm_set_leaves(b->inst[i], snap[i].n, snap[i].k, snap[i].l, snap[i].f, 1);
      if (r != MR_OK) return r;
    }
    return cudaStreamSynchronize(b->st) == cudaSuccess ? MR_OK : MR_ECUDA;
  };
  auto body = [b]() { run_batch_step(b); };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    release();
    return MR_ECUDA;
  }
  // one trial: the snapshot, a step that captures the graphs, then the timed steps
  auto trial = [&](double* ms) -> mr_status {
    mr_status r = restore();
    if (r != MR_OK) return r;
    drop_graphs(*b);
    queue_steps(*b, 1, body);
    for (mr_lbm* h : b->inst) h->cur = b->cur;
    cudaEventRecord(e0, b->st);
    queue_steps(*b, trial_steps, body);
    cudaEventRecord(e1, b->st);
    for (mr_lbm* h : b->inst) h->cur = b->cur;
    if (cudaEventSynchronize(e1) != cudaSuccess) return MR_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return MR_ECUDA;
    for (mr_lbm* h : b->inst) {
      MeshCounts hc[2];
      r = read_counts(h, hc);
      if (r != MR_OK) return r;
    }
    *ms = t / trial_steps;
    return MR_OK;
  };
  // coordinate descent: one phase of one part at a time over the candidates,
  // keeping a change only if it gains more than 1 % (timing noise)
  static const int cand[] = {1, 2, 4, 8, 16, 32};
  double base = 0.0, best = 0.0;
  st = trial(&base);
  best = base;
  for (size_t p = 0; p < b->parts.size() && st == MR_OK; ++p)
    for (int ph = 0; ph < MR_NPH && st == MR_OK; ++ph) {
      int keep = b->parts[p].G.bps[ph];
      for (int c : cand) {
        if (c == keep) continue;
        b->parts[p].G.bps[ph] = c;
        double ms = 0.0;
        st = trial(&ms);
        if (st != MR_OK) break;
        if (ms < 0.99 * best) {
          best = ms;
          keep = c;
        }
      }
      b->parts[p].G.bps[ph] = keep;
    }
  double tuned = 0.0;
  if (st == MR_OK) st = trial(&tuned);  // the chosen schedule, measured once more
  // the batch as it was: leaves, counters, launch counts, no captured step
  if (st == MR_OK) st = restore();
  for (size_t i = 0; i < ni && st == MR_OK; ++i) {
    mr_lbm* h = b->inst[i];
    MeshCounts hc[2];
    if (cudaMemcpy(hc, h->cntbuf, 2 * sizeof(MeshCounts), cudaMemcpyDeviceToHost) != cudaSuccess) {
      st = MR_ECUDA;
      break;
    }
    for (int m = 0; m < 2; ++m) {
      hc[m].leaf_updates = snap[i].cnt[m].leaf_updates;
      hc[m].steps = snap[i].cnt[m].steps;
    }
    if (cudaMemcpy(h->cntbuf, hc, 2 * sizeof(MeshCounts), cudaMemcpyHostToDevice) != cudaSuccess) st = MR_ECUDA;
    h->launches = snap[i].launches;
  }
  b->launches = launches0;
  drop_graphs(*b);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release();
  if (st != MR_OK) return st;
  store_schedule(b);
  if (ms_fixed) *ms_fixed = base;
  if (ms_tuned) *ms_tuned = tuned;
  return MR_OK;
}

mr_status mr_lbm_batch_destroy(mr_lbm_batch_t b) {
  if (b) free_batch(b);
  return MR_OK;
}

}  // extern "C"

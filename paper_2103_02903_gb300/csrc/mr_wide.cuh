// The prediction operator of half-width s = 2, 3 (Table 1; the
// tensor-product operators of Sec. 4.1 for d = 2, 3), shared by the kernels
// of the wide-stencil step (mr_wide.cu) and the dense reconstruction of the
// exact collision (mr_exact.cu).
#pragma once

#include "mr_schemes.cuh"

// Table 1: coefficient c_a (a = 1..s) of the centred prediction of
// half-width s.
template <int S>
__device__ __forceinline__ double wide_coef(int a) {
  if constexpr (S == 2) return a == 1 ? -22.0 / 128.0 : 3.0 / 128.0;
  return a == 1 ? -201.0 / 1024.0 : (a == 2 ? 11.0 / 256.0 : -5.0 / 1024.0);
}

// Arithmetic of the prediction: rounded as written, never contracted
// (EXACT, FP64: the decision path), or plain operators in C.
template <class C, bool EXACT>
struct WAr {
  __device__ static C add(C a, C b) { return a + b; }
  __device__ static C sub(C a, C b) { return a - b; }
  __device__ static C mul(C a, C b) { return a * b; }
};
template <>
struct WAr<double, true> {
  __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ static double sub(double a, double b) { return __dsub_rn(a, b); }
  __device__ static double mul(double a, double b) { return __dmul_rn(a, b); }
};

template <int D, int S>
struct WBox {
  static constexpr int W1 = 2 * S + 1;
  static constexpr int N = D == 1 ? W1 : D == 2 ? W1 * W1 : W1 * W1 * W1;
  // box index of offset (a, b, c), x fastest
  __device__ static constexpr int at(int a, int b, int c) {
    return D == 1 ? a + S : D == 2 ? (b + S) * W1 + (a + S) : ((c + S) * W1 + (b + S)) * W1 + (a + S);
  }
};

// Predicted value of child ci (x bit | y bit << 1 | z bit << 2) from the
// (2s+1)^D stencil v (x fastest): the value of the centre, then the signed
// axis sums sum_a c_a (v_a - v_-a), then the pair sums sum_{b, a} c_a c_b
// times the signed corner combination (b outer, a inner), then in 3D the
// triple sum; the pair terms carry cross_sign.  Every product of a sign
// +-1 is exact, so t + s q is formed as t + q or t - q.
template <int D, int S, class C, bool EXACT>
__device__ __forceinline__ C wide_predict(const C* v, int ci, int cross_sign) {
  using A = WAr<C, EXACT>;
  using B = WBox<D, S>;
  auto V = [&](int a, int b, int c) { return v[B::at(a, b, c)]; };
  auto pm = [](C t, int s, C q) { return s > 0 ? A::add(t, q) : A::sub(t, q); };
  const int sx = (ci & 1) ? -1 : 1, sy = (ci & 2) ? -1 : 1, sz = (ci & 4) ? -1 : 1;
  C q[3];
#pragma unroll
  for (int ax = 0; ax < D; ++ax) {
    auto Va = [&](int o) { return ax == 0 ? V(o, 0, 0) : ax == 1 ? V(0, o, 0) : V(0, 0, o); };
    C acc = A::mul((C)wide_coef<S>(1), A::sub(Va(1), Va(-1)));
#pragma unroll
    for (int a = 2; a <= S; ++a) acc = A::add(acc, A::mul((C)wide_coef<S>(a), A::sub(Va(a), Va(-a))));
    q[ax] = acc;
  }
  C t = V(0, 0, 0);
  t = pm(t, sx, q[0]);
  if constexpr (D == 1) return t;
  t = pm(t, sy, q[1]);
  if constexpr (D == 3) t = pm(t, sz, q[2]);
  // pair sums: (x, y), then in 3D (x, z) and (y, z)
  constexpr int NP = D == 2 ? 1 : 3;
#pragma unroll
  for (int pr = 0; pr < NP; ++pr) {
    C acc = (C)0;
#pragma unroll
    for (int b = 1; b <= S; ++b)
#pragma unroll
      for (int a = 1; a <= S; ++a) {
        auto P = [&](int u, int w) { return pr == 0 ? V(u, w, 0) : pr == 1 ? V(u, 0, w) : V(0, u, w); };
        const C cc = (C)(wide_coef<S>(a) * wide_coef<S>(b));  // exact: short dyadic rationals
        const C term = A::mul(cc, A::add(A::sub(A::sub(P(a, b), P(-a, b)), P(a, -b)), P(-a, -b)));
        acc = (a == 1 && b == 1) ? term : A::add(acc, term);
      }
    const int s1 = pr == 0 ? sx : (pr == 1 ? sx : sy), s2 = pr == 0 ? sy : sz;
    t = pm(t, cross_sign * s1 * s2, acc);
  }
  if constexpr (D == 3) {
    C acc = (C)0;
#pragma unroll
    for (int e = 1; e <= S; ++e)
#pragma unroll
      for (int b = 1; b <= S; ++b)
#pragma unroll
        for (int a = 1; a <= S; ++a) {
          const C ccc = (C)(wide_coef<S>(a) * wide_coef<S>(b) * wide_coef<S>(e));  // exact
          C w = A::sub(V(a, b, e), V(-a, b, e));
          w = A::sub(w, V(a, -b, e));
          w = A::sub(w, V(a, b, -e));
          w = A::add(w, V(-a, -b, e));
          w = A::add(w, V(-a, b, -e));
          w = A::add(w, V(a, -b, -e));
          w = A::sub(w, V(-a, -b, -e));
          const C term = A::mul(ccc, w);
          acc = (a == 1 && b == 1 && e == 1) ? term : A::add(acc, term);
        }
    t = pm(t, sx * sy * sz, acc);
  }
  return t;
}


// Lattice-Boltzmann schemes of the library (velocities, moments, collision,
// equilibria) and the small device helpers that the transport, the ghost
// prediction and the adjoint share.  Every function is a template on the
// arithmetic type C (double, float, or the dual numbers of the adjoint).
#pragma once

#include "mr_common.cuh"

namespace {

// Relaxation rate s[i] in the arithmetic C (the adjoint's dual numbers seed
// it as an independent variable).
template <class C>
struct RateOf {
  __device__ static C get(const Geo& g, int i) { return MR_K(C, g, s[i]); }
};
template <class C>
__device__ __forceinline__ C mr_rate(const Geo& g, int i) {
  return RateOf<C>::get(g, i);
}

template <int S>
struct Scheme;

// D1Q2: eta = (+1, -1), M = [[1, 1], [l, -l]], S = diag(0, s)
template <>
struct Scheme<0> {
  static constexpr int D = 1, Q = 2;
  static constexpr int NR = 1;  // relaxation-rate slots used
  static constexpr bool DIAG = false;
  __device__ static int axis(int p) { return 0; }
  __device__ static int sign(int p) { return p == 0 ? 1 : -1; }
  __device__ static int opp(int p) { return 1 - p; }
  template <class C>
  __device__ static C meq1(const Geo& g, C m0) { return MR_K(C, g, phys[0]) * m0; }
  template <class C>
  __device__ static void collide(const Geo& g, C* f) {
    const C L = MR_K(C, g, lambda), s = mr_rate<C>(g, 0);
    const C m0 = f[0] + f[1];
    C m1 = L * (f[0] - f[1]);
    m1 = ((C)1 - s) * m1 + s * meq1<C>(g, m0);
    f[0] = (C)0.5 * (m0 + m1 / L);
    f[1] = (C)0.5 * (m0 - m1 / L);
  }
  template <class T>
  __device__ static void equilibrium(const Geo& g, const T* u, T* f) {
    const T m1 = meq1<T>(g, u[0]);
    f[0] = (T)0.5 * (u[0] + m1 / (T)g.lambda);
    f[1] = (T)0.5 * (u[0] - m1 / (T)g.lambda);
  }
};

// D1Q2 Burgers: m^eq_1 = u^2 / 2
template <>
struct Scheme<1> : Scheme<0> {
  template <class C>
  __device__ static C meq1(const Geo&, C m0) { return (C)0.5 * m0 * m0; }
  template <class C>
  __device__ static void collide(const Geo& g, C* f) {
    const C L = MR_K(C, g, lambda), s = mr_rate<C>(g, 0);
    const C m0 = f[0] + f[1];
    C m1 = L * (f[0] - f[1]);
    m1 = ((C)1 - s) * m1 + s * meq1<C>(g, m0);
    f[0] = (C)0.5 * (m0 + m1 / L);
    f[1] = (C)0.5 * (m0 - m1 / L);
  }
  template <class T>
  __device__ static void equilibrium(const Geo& g, const T* u, T* f) {
    const T m1 = meq1<T>(g, u[0]);
    f[0] = (T)0.5 * (u[0] + m1 / (T)g.lambda);
    f[1] = (T)0.5 * (u[0] - m1 / (T)g.lambda);
  }
};

// D1Q3 shallow water: eta = (0, +1, -1), M = [[1,1,1],[0,l,-l],[0,l^2,l^2]]
template <>
struct Scheme<2> {
  static constexpr int D = 1, Q = 3;
  static constexpr int NR = 1;
  static constexpr bool DIAG = false;
  __device__ static int axis(int p) { return p == 0 ? -1 : 0; }
  __device__ static int sign(int p) { return p == 1 ? 1 : -1; }
  __device__ static int opp(int p) { return p == 0 ? 0 : 3 - p; }
  template <class C>
  __device__ static void collide(const Geo& g, C* f) {
    const C L = MR_K(C, g, lambda), s = mr_rate<C>(g, 0), gr = MR_K(C, g, phys[0]);
    const C m0 = f[0] + f[1] + f[2];
    const C m1 = L * (f[1] - f[2]);
    C m2 = L * L * (f[1] + f[2]);
    m2 = ((C)1 - s) * m2 + s * (m1 * m1 / m0 + (C)0.5 * gr * m0 * m0);
    const C t = m2 / (L * L);
    f[0] = m0 - t;
    f[1] = (C)0.5 * (t + m1 / L);
    f[2] = (C)0.5 * (t - m1 / L);
  }
  template <class T>
  __device__ static void equilibrium(const Geo& g, const T* u, T* f) {
    const T L = (T)g.lambda;
    const T t = (u[1] * u[1] / u[0] + (T)0.5 * (T)g.phys[0] * u[0] * u[0]) / (L * L);
    f[0] = u[0] - t;
    f[1] = (T)0.5 * (t + u[1] / L);
    f[2] = (T)0.5 * (t - u[1] / L);
  }
};

// D2Q4^4 Euler: per lattice i, eta = (1,0), (0,1), (-1,0), (0,-1)
template <>
struct Scheme<3> {
  static constexpr int D = 2, Q = 16;
  static constexpr int NR = 8;
  static constexpr bool DIAG = false;
  __device__ static int axis(int p) { return (p & 3) & 1; }
  __device__ static int sign(int p) { return (p & 3) < 2 ? 1 : -1; }
  __device__ static int opp(int p) { return (p & ~3) | ((p + 2) & 3); }
  template <class C>
  __device__ static void fluxes(const Geo& g, const C* u, C* fx, C* fy) {
    const C rho = u[0], mx = u[1], my = u[2], E = u[3], gam = MR_K(C, g, phys[0]);
    const C irho = (C)1 / rho;  // one division per cell
    const C vx = mx * irho, vy = my * irho;
    const C pr = (gam - (C)1) * (E - (C)0.5 * (mx * vx + my * vy));
    fx[0] = mx; fx[1] = mx * vx + pr; fx[2] = my * vx; fx[3] = vx * (E + pr);
    fy[0] = my; fy[1] = mx * vy; fy[2] = my * vy + pr; fy[3] = vy * (E + pr);
  }
  template <class C>
  __device__ static void from_moments(const Geo& g, C m0, C m1, C m2, C m3, C* f) {
    const C il = MR_K(C, g, inv_lambda), il2 = il * il;
    const C a = (C)0.25 * m0, b = (C)0.5 * m1 * il, c = (C)0.5 * m2 * il, e = (C)0.25 * m3 * il2;
    f[0] = a + b + e;
    f[1] = a + c - e;
    f[2] = a - b + e;
    f[3] = a - c - e;
  }
  template <class C>
  __device__ static void collide(const Geo& g, C* f) {
    const C L = MR_K(C, g, lambda);
    C m[4][4], u[4], fx[4], fy[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const C* fi = f + 4 * i;
      m[i][0] = fi[0] + fi[1] + fi[2] + fi[3];
      m[i][1] = L * (fi[0] - fi[2]);
      m[i][2] = L * (fi[1] - fi[3]);
      m[i][3] = L * L * (fi[0] - fi[1] + fi[2] - fi[3]);
      u[i] = m[i][0];
    }
    fluxes<C>(g, u, fx, fy);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const C sq = mr_rate<C>(g, i), sxy = mr_rate<C>(g, 4 + i);
      const C m1 = ((C)1 - sq) * m[i][1] + sq * fx[i];
      const C m2 = ((C)1 - sq) * m[i][2] + sq * fy[i];
      const C m3 = ((C)1 - sxy) * m[i][3];
      from_moments<C>(g, m[i][0], m1, m2, m3, f + 4 * i);
    }
  }
  template <class T>
  __device__ static void equilibrium(const Geo& g, const T* u, T* f) {
    T fx[4], fy[4];
    fluxes<T>(g, u, fx, fy);
#pragma unroll
    for (int i = 0; i < 4; ++i) from_moments<T>(g, u[i], fx[i], fy[i], (T)0.0, f + 4 * i);
  }
};

// nine small integers (t + bias, each below 2^bits) packed into one word
struct MrNine {
  int v[9];
};
__host__ __device__ constexpr unsigned long long mr_pack9(MrNine t, int bias, int bits) {
  unsigned long long r = 0;
  for (int i = 0; i < 9; ++i) r |= (unsigned long long)(t.v[i] + bias) << (bits * i);
  return r;
}

// D2Q9 of Sec. 7.2.2: eta^0 = 0, eta^{1..4} = (1,0), (0,1), (-1,0), (0,-1),
// eta^{5..8} = (1,1), (-1,1), (-1,-1), (1,-1).  The rows of M are mutually
// orthogonal; divided by their power of lambda they are the integer rows
// R_r below, so M^{-1} = M^T diag(1/|row|^2) and, with j = q / lambda, the
// equilibria of the scaled moments mu_r = R_r . f carry no lambda.
template <>
struct Scheme<4> {
  static constexpr int D = 2, Q = 9;
  static constexpr int NR = 2;
  static constexpr bool DIAG = true;
  static constexpr int DIAG0 = 5;  // first diagonal population
  // velocities and opposites packed into integer constants (2 and 4 bits
  // per population), so that a population index known only at run time
  // needs no table in memory
  static constexpr uint32_t EXP = (uint32_t)mr_pack9({0, 1, 0, -1, 0, 1, -1, -1, 1}, 1, 2);
  static constexpr uint32_t EYP = (uint32_t)mr_pack9({0, 0, 1, 0, -1, 1, 1, -1, -1}, 1, 2);
  static constexpr unsigned long long OPPP = mr_pack9({0, 3, 4, 1, 2, 7, 8, 5, 6}, 0, 4);
  __device__ static int eta(int p, int a) { return (int)(((a == 0 ? EXP : EYP) >> (2 * p)) & 3u) - 1; }
  __device__ static int opp(int p) { return (int)((OPPP >> (4 * p)) & 15ull); }
  // f = sum_r R_r mu_r / |R_r|^2
  template <class C>
  __device__ static void from_moments(const C* mu, C* f) {
    const C a0 = mu[0] / (C)9, a1 = mu[1] / (C)6, a2 = mu[2] / (C)6, a3 = mu[3] / (C)36;
    const C a4 = mu[4] / (C)12, a5 = mu[5] / (C)12, a6 = mu[6] / (C)36, a7 = mu[7] / (C)4, a8 = mu[8] / (C)4;
    const C b = a0 - a3 - (C)2 * a6;      // axis populations, common part
    const C c = a0 + (C)2 * a3 + a6;      // diagonal populations, common part
    f[0] = a0 - (C)4 * a3 + (C)4 * a6;
    f[1] = b + a1 - (C)2 * a4 + a7;
    f[2] = b + a2 - (C)2 * a5 - a7;
    f[3] = b - a1 + (C)2 * a4 + a7;
    f[4] = b - a2 + (C)2 * a5 - a7;
    f[5] = c + a1 + a2 + a4 + a5 + a8;
    f[6] = c - a1 + a2 - a4 + a5 - a8;
    f[7] = c - a1 - a2 - a4 - a5 + a8;
    f[8] = c + a1 - a2 + a4 - a5 - a8;
  }
  // equilibria of mu_3 .. mu_8 (energy, heat fluxes, energy square, stresses)
  template <class C>
  __device__ static void equilibria(C rho, C jx, C jy, C* mu) {
    const C ir = (C)1 / rho;
    const C j2 = (jx * jx + jy * jy) * ir;
    mu[3] = (C)-2 * rho + (C)3 * j2;
    mu[4] = -jx;
    mu[5] = -jy;
    mu[6] = rho - (C)3 * j2;
    mu[7] = (jx * jx - jy * jy) * ir;
    mu[8] = jx * jy * ir;
  }
  template <class C>
  __device__ static void collide(const Geo& g, C* f) {
    const C s14 = (f[1] + f[2]) + (f[3] + f[4]), s58 = (f[5] + f[6]) + (f[7] + f[8]);
    const C dx1 = f[1] - f[3], dy1 = f[2] - f[4];
    const C dx2 = (f[5] - f[7]) + (f[8] - f[6]), dy2 = (f[5] - f[7]) + (f[6] - f[8]);
    C mu[9], eq[9];
    mu[0] = f[0] + s14 + s58;
    mu[1] = dx1 + dx2;
    mu[2] = dy1 + dy2;
    mu[3] = (C)-4 * f[0] - s14 + (C)2 * s58;
    mu[4] = (C)-2 * dx1 + dx2;
    mu[5] = (C)-2 * dy1 + dy2;
    mu[6] = (C)4 * f[0] - (C)2 * s14 + s58;
    mu[7] = (f[1] - f[2]) + (f[3] - f[4]);
    mu[8] = (f[5] - f[6]) + (f[7] - f[8]);
    equilibria<C>(mu[0], mu[1], mu[2], eq);
    const C s1 = mr_rate<C>(g, 0), s2 = mr_rate<C>(g, 1);
#pragma unroll
    for (int r = 3; r < 9; ++r) {
      const C s = r < 7 ? s1 : s2;
      mu[r] = ((C)1 - s) * mu[r] + s * eq[r];
    }
    from_moments<C>(mu, f);
  }
  template <class T>
  __device__ static void equilibrium(const Geo& g, const T* u, T* f) {
    T mu[9];
    mu[0] = u[0];
    mu[1] = u[1] * (T)g.inv_lambda;
    mu[2] = u[2] * (T)g.inv_lambda;
    equilibria<T>(mu[0], mu[1], mu[2], mu);
    from_moments<T>(mu, f);
  }
};

// D3Q6 advection (Sec. 7.3): eta = +-e_x, +-e_y, +-e_z, the printed M,
// S = diag(0, s1, s1, s1, s2, s2), m^eq = (u, V_x u, V_y u, V_z u, 0, 0).
// With a = f0 + f1, b = f2 + f3, c = f4 + f5 the even rows are
// m0 = a + b + c, m4 = l^2 (a - b), m5 = l^2 (a - c), so M^-1 is closed form.
template <>
struct Scheme<5> {
  static constexpr int D = 3, Q = 6;
  static constexpr int NR = 2;
  static constexpr bool DIAG = false;
  __device__ static int axis(int p) { return p >> 1; }
  __device__ static int sign(int p) { return (p & 1) ? -1 : 1; }
  __device__ static int opp(int p) { return p ^ 1; }
  template <class C>
  __device__ static void from_moments(const Geo& g, const C* m, C* f) {
    const C il = MR_K(C, g, inv_lambda), il2 = il * il;
    const C a = (m[0] + (m[4] + m[5]) * il2) / (C)3;
    const C b = a - m[4] * il2, c = a - m[5] * il2;
    f[0] = (C)0.5 * (a + m[1] * il);
    f[1] = (C)0.5 * (a - m[1] * il);
    f[2] = (C)0.5 * (b + m[2] * il);
    f[3] = (C)0.5 * (b - m[2] * il);
    f[4] = (C)0.5 * (c + m[3] * il);
    f[5] = (C)0.5 * (c - m[3] * il);
  }
  template <class C>
  __device__ static void collide(const Geo& g, C* f) {
    const C L = MR_K(C, g, lambda), L2 = L * L;
    const C s1 = mr_rate<C>(g, 0), s2 = mr_rate<C>(g, 1);
    C m[6];
    const C a = f[0] + f[1], b = f[2] + f[3], c = f[4] + f[5];
    m[0] = a + b + c;
    m[1] = L * (f[0] - f[1]);
    m[2] = L * (f[2] - f[3]);
    m[3] = L * (f[4] - f[5]);
    m[4] = L2 * (a - b);
    m[5] = L2 * (a - c);
#pragma unroll
    for (int r = 1; r <= 3; ++r) m[r] = ((C)1 - s1) * m[r] + s1 * (MR_K(C, g, phys[r - 1]) * m[0]);
    m[4] = ((C)1 - s2) * m[4];
    m[5] = ((C)1 - s2) * m[5];
    from_moments<C>(g, m, f);
  }
  template <class T>
  __device__ static void equilibrium(const Geo& g, const T* u, T* f) {
    T m[6] = {u[0], (T)g.phys[0] * u[0], (T)g.phys[1] * u[0], (T)g.phys[2] * u[0], (T)0, (T)0};
    const T il = (T)g.inv_lambda, il2 = il * il;
    const T a = (m[0] + (m[4] + m[5]) * il2) / (T)3;
    const T b = a - m[4] * il2, c = a - m[5] * il2;
    f[0] = (T)0.5 * (a + m[1] * il);
    f[1] = (T)0.5 * (a - m[1] * il);
    f[2] = (T)0.5 * (b + m[2] * il);
    f[3] = (T)0.5 * (b - m[2] * il);
    f[4] = (T)0.5 * (c + m[3] * il);
    f[5] = (T)0.5 * (c - m[3] * il);
  }
};

// eta^p_a in {-1, 0, 1} of the schemes with axis velocities only
template <class Sc>
__device__ __forceinline__ int eta_of(int p, int a) {
  if constexpr (Sc::DIAG)
    return Sc::eta(p, a);
  else
    return Sc::axis(p) == a ? Sc::sign(p) : 0;
}

template <class C>
__device__ __forceinline__ C bc_value(const Geo& g, int kind, const C* f, int p, int pd) {
  switch (kind) {
    case 1: return f[p];                    // copy
    case 2: return f[pd];                   // bounce back
    case 3: return -f[pd];                  // anti bounce back
    case 4: return f[pd] + MR_K(C, g, bcv[p]);     // bounce back with the wall velocity u0
    default: return (C)0;
  }
}

// s = 1 prediction in arithmetic C (contraction allowed; off the decision path)
template <int D, class C>
__device__ __forceinline__ C predict_c(const C* v, int ci, C cross_sign) {
  const C sx = (ci & 1) ? (C)-1 : (C)1;
  const C c1 = (C)MR_C1;
  if constexpr (D == 1) {
    return v[1] + sx * (c1 * (v[2] - v[0]));
  } else if constexpr (D == 3) {
#define MR_V3(a, b, c) v[(((c) + 1) * 3 + ((b) + 1)) * 3 + ((a) + 1)]
    const C sy = (ci & 2) ? (C)-1 : (C)1, sz = (ci & 4) ? (C)-1 : (C)1;
    const C qx = c1 * (MR_V3(1, 0, 0) - MR_V3(-1, 0, 0));
    const C qy = c1 * (MR_V3(0, 1, 0) - MR_V3(0, -1, 0));
    const C qz = c1 * (MR_V3(0, 0, 1) - MR_V3(0, 0, -1));
    const C qxy = (c1 * c1) * (((MR_V3(1, 1, 0) - MR_V3(-1, 1, 0)) - MR_V3(1, -1, 0)) + MR_V3(-1, -1, 0));
    const C qxz = (c1 * c1) * (((MR_V3(1, 0, 1) - MR_V3(-1, 0, 1)) - MR_V3(1, 0, -1)) + MR_V3(-1, 0, -1));
    const C qyz = (c1 * c1) * (((MR_V3(0, 1, 1) - MR_V3(0, -1, 1)) - MR_V3(0, 1, -1)) + MR_V3(0, -1, -1));
    const C q3 = (c1 * c1 * c1) * (((((((MR_V3(1, 1, 1) - MR_V3(-1, 1, 1)) - MR_V3(1, -1, 1)) - MR_V3(1, 1, -1)) +
                                       MR_V3(-1, -1, 1)) + MR_V3(-1, 1, -1)) + MR_V3(1, -1, -1)) -
                                    MR_V3(-1, -1, -1));
    const C t = MR_V3(0, 0, 0);
#undef MR_V3
    return t + sx * qx + sy * qy + sz * qz + (cross_sign * sx * sy) * qxy + (cross_sign * sx * sz) * qxz +
           (cross_sign * sy * sz) * qyz + (sx * sy * sz) * q3;
  } else {
    const C sy = (ci & 2) ? (C)-1 : (C)1;
    const C qx = c1 * (v[5] - v[3]);
    const C qy = c1 * (v[7] - v[1]);
    const C q2 = (c1 * c1) * (((v[8] - v[6]) - v[2]) + v[0]);
    return v[4] + sx * qx + sy * qy + (cross_sign * sx * sy) * q2;
  }
}

// Coefficients of the 3^D stencil values (x fastest) in the prediction of
// child ci: the same operator as predict_c, written as its weights.
template <int D>
__device__ __forceinline__ void predict_weights(int ci, double cross_sign, double* w) {
  const double sx = (ci & 1) ? -1.0 : 1.0, c1 = MR_C1;
  if (D == 1) {
    w[0] = -sx * c1;
    w[1] = 1.0;
    w[2] = sx * c1;
  } else {
    const double sy = (ci & 2) ? -1.0 : 1.0, q = cross_sign * sx * sy * c1 * c1;
    w[0] = q;
    w[1] = -sy * c1;
    w[2] = -q;
    w[3] = -sx * c1;
    w[4] = 1.0;
    w[5] = sx * c1;
    w[6] = -q;
    w[7] = sy * c1;
    w[8] = q;
  }
}

template <class C, class S>
__device__ __forceinline__ C ld_c(const ValPtr<S>& v, int p) {
  return (C)mr_cvt_d(__ldg(v.p + (size_t)p * v.stride));
}
template <>
__device__ __forceinline__ float ld_c<float, float>(const ValPtr<float>& v, int p) {
  return __ldg(v.p + (size_t)p * v.stride);
}
template <>
__device__ __forceinline__ float ld_c<float, __half>(const ValPtr<__half>& v, int p) {
  return __half2float(__ldg(v.p + (size_t)p * v.stride));
}
template <>
__device__ __forceinline__ float ld_c<float, __nv_bfloat16>(const ValPtr<__nv_bfloat16>& v, int p) {
  return __bfloat162float(__ldg(v.p + (size_t)p * v.stride));
}

// Value of population p as arithmetic C, with the storage offset added back
// in the 16-bit forms (no arithmetic at all in the others).
template <int F>
__device__ __forceinline__ typename FormT<F>::C ld_off(const ValPtr<typename FormT<F>::S>& v, int p,
                                                       const typename FormT<F>::C* offv) {
  using C = typename FormT<F>::C;
  if constexpr (FormT<F>::offs)
    return ld_c<C>(v, p) + offv[p];
  else
    return ld_c<C>(v, p);
}

// finiteness from the exponent bits (integer pipe, not the FP64 one)
__device__ __forceinline__ bool is_finite_bits(double x) {
  return (__double_as_longlong(x) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool is_finite_bits(float x) { return (__float_as_int(x) & 0x7f800000) != 0x7f800000; }

// Weight of the level-(l+1) cell 2k + r in the incoming-minus-outgoing
// finest values of the leaf k along axis a, for the velocity sign s:
// s > 0: R_{2k-1} - R_{2k+1} (the finest cell upwind of the leaf and the
// leaf's last finest cell), s < 0: L_{2k+2} - L_{2k}.  The upwind term is
// absent at a non-periodic boundary (that cell is outside the domain).
template <class C>
__device__ __forceinline__ C corner_edge_weight(const Geo& g, const C* __restrict__ W, int l1, int a, int k,
                                                     int r, int s) {
  const int per = g.periodic[a], N1 = g.n[l1][a], N = g.n[l1 - 1][a];
  const int tab = s > 0 ? 2 : 3;
  const int cu = s > 0 ? 2 * k - 1 : 2 * k + 2, co = s > 0 ? 2 * k + 1 : 2 * k;
  const int du = 2 * k + r - cu, dd = 2 * k + r - co;
  C w = (C)0;
  if ((per || (s > 0 ? k > 0 : k < N - 1)) && du >= -2 && du <= 2)
    w += W[MR_WIDX(l1, a, mr_slot(per ? 2 : cu, N1, per), tab) + du + 2];
  if (dd >= -2 && dd <= 2) w -= W[MR_WIDX(l1, a, mr_slot(per ? 2 : co, N1, per), tab) + dd + 2];
  return w;
}

// Obstacle fraction of a leaf (Sec. 7.2.2): the share of its finest-cell
// centres inside the disc, each centre tested with the FP64 operations of
// the plain definition in the same order (no contraction).  The rounded
// squared distance is unimodal along a row of centres, so the centres of a
// row inside the disc are one range: found from the column nearest to the
// disc centre by bisection on either side.
__device__ __forceinline__ bool in_disc(const Geo& g, long long ix, double ey2) {
  const double xc = __dadd_rn(g.xlo[0], __dmul_rn((double)ix + 0.5, g.dxJ));
  const double ex = __dsub_rn(xc, g.obs[0]);
  return __dadd_rn(__dmul_rn(ex, ex), ey2) <= __dmul_rn(g.obs[2], g.obs[2]);
}

__device__ double obstacle_fraction(const Geo& g, int l, uint32_t code) {
  int kx, ky;
  mr_decode(g, l, code, kx, ky);
  const int w = 1 << (g.J - l);
  const long long x0 = (long long)kx * w, y0 = (long long)ky * w;
  const double h = g.dxJ, m = g.obs[2] + 2.0 * h;
  if (g.xlo[0] + (double)(x0 + w) * h < g.obs[0] - m || g.xlo[0] + (double)x0 * h > g.obs[0] + m ||
      g.xlo[1] + (double)(y0 + w) * h < g.obs[1] - m || g.xlo[1] + (double)y0 * h > g.obs[1] + m)
    return 0.0;
  long long cc = __double2ll_rn((g.obs[0] - g.xlo[0]) / h - 0.5) - x0;
  cc = cc < 0 ? 0 : (cc > w - 1 ? w - 1 : cc);
  long long inside = 0;
  for (int by = 0; by < w; ++by) {
    const double yc = __dadd_rn(g.xlo[1], __dmul_rn((double)(y0 + by) + 0.5, h));
    const double ey = __dsub_rn(yc, g.obs[1]);
    const double ey2 = __dmul_rn(ey, ey);
    long long c = -1;
    for (long long t = cc - 1; t <= cc + 1; ++t)
      if (t >= 0 && t < w && in_disc(g, x0 + t, ey2)) {
        c = t;
        break;
      }
    if (c < 0) continue;
    long long lo = 0, hi = c;  // first centre inside
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (in_disc(g, x0 + mid, ey2))
        hi = mid;
      else
        lo = mid + 1;
    }
    const long long first = lo;
    lo = c;
    hi = w - 1;  // last centre inside
    while (lo < hi) {
      const long long mid = (lo + hi + 1) >> 1;
      if (in_disc(g, x0 + mid, ey2))
        lo = mid;
      else
        hi = mid - 1;
    }
    inside += lo - first + 1;
  }
  return inside ? (double)inside / ((double)w * (double)w) : 0.0;
}

template <int Q>
struct PopRows {
  static constexpr int value = Q < 8 ? Q : 8;
};

}  // namespace

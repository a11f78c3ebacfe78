// Velocity sets as compile-time structure (Sec. 2.1: D2Q9; Sec. 3.2: a
// 13-velocity 3D set, read as rest + icosahedron vertices, |e| = sqrt(5/3);
// the cubic D3Q19 and D3Q27 as alternatives).
//
// Velocities are e_a = S * C_a with C_a built from 0, +-1 and +-phi, ordered
// so that a's opposite is known at compile time.  The helpers below contract
// e_a with a vector using only the non-zero components (FP64 is the scarce
// resource on B300, so multiplications by 0 or 1 are never issued).
#pragma once

namespace semlbm {

constexpr double kPhi = 1.618033988749895;          // golden ratio
constexpr double kCs2 = 1.0 / 3.0;                  // c_s^2 for both sets
constexpr double kInvCs2 = 3.0;

struct D2Q9 {
  static constexpr int D = 2, Q = 9, NREP = 4;
  static constexpr bool PAIR_METRIC = false;   // pair coefficients cost 0-2 adds: computed
  // streaming derivative chains start from t v (4 FP64 operations fewer per pair)
  static constexpr bool TV_START = true;
  static constexpr double S = 1.0;                   // |C| -> |e| scale
  static constexpr double SPEED_MAX = 1.4142135623730951;
  __host__ __device__ static constexpr int rep(int r) { return r < 2 ? 1 + r : 3 + r; }   // 1,2,5,6
  __host__ __device__ static constexpr int opp(int a) {
    return a == 0 ? 0 : (a <= 4 ? (a <= 2 ? a + 2 : a - 2) : (a <= 6 ? a + 2 : a - 2));
  }
  __host__ __device__ static constexpr double t(int a) {
    return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  // component c of C_a (host tables and tests)
  __host__ __device__ static constexpr double C(int a, int c) {
    constexpr int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    return c == 0 ? ex[a] : (c == 1 ? ey[a] : 0);
  }
  // C_a . v for a representative a in {1,2,5,6}
  template <int A>
  __device__ static __forceinline__ double cdot(const double* v) {
    if constexpr (A == 1) return v[0];
    else if constexpr (A == 2) return v[1];
    else if constexpr (A == 5) return v[0] + v[1];
    else return v[1] - v[0];                         // A == 6: (-1, 1)
  }
};

struct D3Q13 {
  static constexpr int D = 3, Q = 13, NREP = 6;
  static constexpr bool PAIR_METRIC = true;    // pair coefficients cost 3 fma: stored per node
  static constexpr bool TV_START = true;       // one moving weight: t v formed once per node
  static constexpr double S = 0.6787159472735029;    // sqrt(5/3) / sqrt(1 + phi^2)
  static constexpr double SPEED_MAX = 1.2909944487358056;
  __host__ __device__ static constexpr int rep(int r) { return 1 + r; }  // 1..6, opp = a + 6
  __host__ __device__ static constexpr int opp(int a) { return a == 0 ? 0 : (a <= 6 ? a + 6 : a - 6); }
  __host__ __device__ static constexpr double t(int a) { return a == 0 ? 0.4 : 0.05; }
  __host__ __device__ static constexpr double C(int a, int c) {
    constexpr double tab[7][3] = {{0, 0, 0},     {0, 1, kPhi},  {0, -1, kPhi}, {1, kPhi, 0},
                                  {-1, kPhi, 0}, {kPhi, 0, 1},  {kPhi, 0, -1}};
    return a <= 6 ? tab[a][c] : -tab[a - 6][c];
  }
  template <int A>
  __device__ static __forceinline__ double cdot(const double* v) {
    if constexpr (A == 1) return fma(kPhi, v[2], v[1]);
    else if constexpr (A == 2) return fma(kPhi, v[2], -v[1]);
    else if constexpr (A == 3) return fma(kPhi, v[1], v[0]);
    else if constexpr (A == 4) return fma(kPhi, v[1], -v[0]);
    else if constexpr (A == 5) return fma(kPhi, v[0], v[2]);
    else return fma(kPhi, v[0], -v[2]);              // A == 6
  }
};

// C . v for an integer velocity C with components in {-1, 0, 1} and a positive
// first non-zero component (the representatives of the cubic sets below)
template <int C0, int C1, int C2>
__device__ __forceinline__ double idot3(const double* v) {
  double r;
  if constexpr (C0 != 0) {
    r = v[0];
    if constexpr (C1 > 0) r += v[1];
    else if constexpr (C1 < 0) r -= v[1];
    if constexpr (C2 > 0) r += v[2];
    else if constexpr (C2 < 0) r -= v[2];
  } else if constexpr (C1 != 0) {
    r = v[1];
    if constexpr (C2 > 0) r += v[2];
    else if constexpr (C2 < 0) r -= v[2];
  } else {
    r = v[2];
  }
  return r;
}

// representatives of the cubic sets: faces, edges, corners
__host__ __device__ constexpr int cubic_rep(int r, int c) {
  constexpr int tab[13][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1},  {1, 1, 0},  {1, -1, 0},
                              {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}, {1, 1, 1},
                              {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
  return tab[r][c];
}

// D3Q19 and D3Q27: cubic velocity sets (c_s^2 = 1/3), e_{a+H} = -e_a
template <int NR>
struct Cubic {
  static constexpr int D = 3, Q = 2 * NR + 1, NREP = NR;
  static constexpr bool PAIR_METRIC = false;
  // two or three moving weights: t v per weight would stay live across the pair
  // loop and spill, so t (c.v) is formed once per pair instead
  static constexpr bool TV_START = false;
  static constexpr double S = 1.0;
  static constexpr double SPEED_MAX = (NR == 9) ? 1.4142135623730951 : 1.7320508075688772;
  __host__ __device__ static constexpr int rep(int r) { return 1 + r; }
  __host__ __device__ static constexpr int opp(int a) { return a == 0 ? 0 : (a <= NR ? a + NR : a - NR); }
  __host__ __device__ static constexpr double t(int a) {
    return NR == 9 ? (a == 0 ? 1.0 / 3.0 : (((a - 1) % 9) < 3 ? 1.0 / 18.0 : 1.0 / 36.0))
                   : (a == 0 ? 8.0 / 27.0
                             : (((a - 1) % 13) < 3 ? 2.0 / 27.0
                                                   : (((a - 1) % 13) < 9 ? 1.0 / 54.0 : 1.0 / 216.0)));
  }
  __host__ __device__ static constexpr double C(int a, int c) {
    return a == 0 ? 0.0 : (a <= NR ? cubic_rep(a - 1, c) : -cubic_rep(a - 1 - NR, c));
  }
  template <int A>
  __device__ static __forceinline__ double cdot(const double* v) {
    return idot3<cubic_rep(A - 1, 0), cubic_rep(A - 1, 1), cubic_rep(A - 1, 2)>(v);
  }
};
using D3Q19 = Cubic<9>;
using D3Q27 = Cubic<13>;

// compile-time loop: f(std::integral_constant<int, I>) for I in [B, E)
template <int I> struct Int { static constexpr int value = I; };
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(Int<B>{});
    static_for<B + 1, E>(f);
  }
}

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

}  // namespace semlbm

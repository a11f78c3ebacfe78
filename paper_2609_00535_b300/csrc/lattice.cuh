// Velocity sets as compile-time structure (Sec. 2.1: D2Q9; Sec. 3.2: a
// 13-velocity 3D set, read as rest + icosahedron vertices, |e| = sqrt(5/3)).
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

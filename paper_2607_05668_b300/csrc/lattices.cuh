// Discrete velocity sets (c_i, w_i, c_s^2) as compile-time tables.
//
// D2Q5 and D3Q7 are the paper's stencils (supplement, stencil table); D2Q9 and D3Q19
// are the standard symmetric sets, admissible because they satisfy the isotropy
// conditions of Sec. 2.2.1.  Population order is this library's own: rest first, then
// axis pairs (+, -), then diagonal pairs (+, -) so that i and its opposite are adjacent.
#pragma once

namespace lbx {

struct LatD2Q5 {
  static constexpr int Q = 5, D = 2, ID = 1;
  __host__ __device__ static constexpr int c(int i, int d) {
    constexpr int C[5][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}};
    return C[i][d];
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
  static constexpr double cs2 = 1.0 / 3.0;
};

struct LatD2Q9 {
  static constexpr int Q = 9, D = 2, ID = 2;
  __host__ __device__ static constexpr int c(int i, int d) {
    constexpr int C[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                             {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    return C[i][d];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  static constexpr double cs2 = 1.0 / 3.0;
};

struct LatD3Q7 {
  static constexpr int Q = 7, D = 3, ID = 3;
  __host__ __device__ static constexpr int c(int i, int d) {
    constexpr int C[7][3] = {{0, 0, 0},  {1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                             {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    return C[i][d];
  }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 0.25 : 0.125; }
  static constexpr double cs2 = 0.25;
};

struct LatD3Q19 {
  static constexpr int Q = 19, D = 3, ID = 4;
  __host__ __device__ static constexpr int c(int i, int d) {
    constexpr int C[19][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                              {0, 0, 1},   {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                              {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                              {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return C[i][d];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  static constexpr double cs2 = 1.0 / 3.0;
};

// The velocity opposite to i (c_opp(i) = -c_i): every set lists rest first, then (+c, -c)
// pairs.  opp_valid() checks that structure at compile time.
template <class Lat>
__host__ __device__ constexpr int opp(int i) {
  return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
}
template <class Lat>
__host__ __device__ constexpr bool opp_valid() {
  for (int i = 0; i < Lat::Q; ++i)
    for (int d = 0; d < 3; ++d)
      if (Lat::c(opp<Lat>(i), d) != -Lat::c(i, d)) return false;
  return true;
}

// Weights for binary32 arithmetic: the moving weights rounded to multiples of 2^-26
// (exact in binary32) and the rest weight 1 minus their sum, so that the weights add up
// to exactly 1.  The nearest binary32 values of 1/3, 1/6, 1/9, ... add up to about
// 1 + 3e-8, and an update that forms w_i (X + ...) would then gain that fraction of X at
// every step: a systematic drift of about 6e-8 of the field per step.  The change of the
// moving weights (at most 2^-27 absolute) is far below the binary32 rounding of the update.
template <class Lat>
__host__ __device__ constexpr double weight_sum1(int i) {
  constexpr double S = 67108864.0;   // 2^26
  if (i != 0) return (double)(long long)(Lat::w(i) * S + 0.5) / S;
  double r = 1.0;
  for (int j = 1; j < Lat::Q; ++j) r -= (double)(long long)(Lat::w(j) * S + 0.5) / S;
  return r;
}

// Lattice weight w_i in the arithmetic type T (binary64: the exact value's nearest double).
template <class Lat, typename T>
__host__ __device__ constexpr T weight(int i) {
  return sizeof(T) == 8 ? T(Lat::w(i)) : T(weight_sum1<Lat>(i));
}

}  // namespace lbx

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

}  // namespace lbx

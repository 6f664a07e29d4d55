// Velocity sets of Sec. 2 ("Velocity stencils", Fig. 1), listed shell by shell. Within a
// 4-member shell the opposite of member k is member k+2, within an 8-member shell it is k+4,
// so the first half of every shell holds one velocity of each +/- pair.
#pragma once

struct D2Q37 {
  static constexpr int Q = 37, M = 3, ORDER = 4, NSHELL = 8;
  __host__ __device__ static constexpr int ex(int i) {
    constexpr int t[37] = {0, 1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0, 2, 1, -1, -2, -2,
                           -1, 1, 2, 2, -2, -2, 2, 3, 0, -3, 0, 3, 1, -1, -3, -3, -1, 1, 3};
    return t[i];
  }
  __host__ __device__ static constexpr int ey(int i) {
    constexpr int t[37] = {0, 0, 1, 0, -1, 1, 1, -1, -1, 0, 2, 0, -2, 1, 2, 2, 1, -1,
                           -2, -2, -1, 2, 2, -2, -2, 0, 3, 0, -3, 1, 3, 3, 1, -1, -3, -3, -1};
    return t[i];
  }
  // shell base vectors (a, b), a >= b >= 0, and their first direction index / size
  __host__ __device__ static constexpr int shell_a(int s) {
    constexpr int t[8] = {0, 1, 1, 2, 2, 2, 3, 3};
    return t[s];
  }
  __host__ __device__ static constexpr int shell_b(int s) {
    constexpr int t[8] = {0, 0, 1, 0, 1, 2, 0, 1};
    return t[s];
  }
  __host__ __device__ static constexpr int shell_first(int s) {
    constexpr int t[8] = {0, 1, 5, 9, 13, 21, 25, 29};
    return t[s];
  }
  __host__ __device__ static constexpr int shell_size(int s) {
    constexpr int t[8] = {1, 4, 4, 4, 8, 4, 4, 8};
    return t[s];
  }
};

struct D2Q17 {
  static constexpr int Q = 17, M = 3, ORDER = 3, NSHELL = 5;
  __host__ __device__ static constexpr int ex(int i) {
    constexpr int t[17] = {0, 1, 0, -1, 0, 1, -1, -1, 1, 2, -2, -2, 2, 3, 0, -3, 0};
    return t[i];
  }
  __host__ __device__ static constexpr int ey(int i) {
    constexpr int t[17] = {0, 0, 1, 0, -1, 1, 1, -1, -1, 2, 2, -2, -2, 0, 3, 0, -3};
    return t[i];
  }
  __host__ __device__ static constexpr int shell_a(int s) {
    constexpr int t[5] = {0, 1, 1, 2, 3};
    return t[s];
  }
  __host__ __device__ static constexpr int shell_b(int s) {
    constexpr int t[5] = {0, 0, 1, 2, 0};
    return t[s];
  }
  __host__ __device__ static constexpr int shell_first(int s) {
    constexpr int t[5] = {0, 1, 5, 9, 13};
    return t[s];
  }
  __host__ __device__ static constexpr int shell_size(int s) {
    constexpr int t[5] = {1, 4, 4, 4, 4};
    return t[s];
  }
};

struct D2Q9 {
  static constexpr int Q = 9, M = 1, ORDER = 2, NSHELL = 3;
  __host__ __device__ static constexpr int ex(int i) {
    constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    return t[i];
  }
  __host__ __device__ static constexpr int ey(int i) {
    constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    return t[i];
  }
  __host__ __device__ static constexpr int shell_a(int s) {
    constexpr int t[3] = {0, 1, 1};
    return t[s];
  }
  __host__ __device__ static constexpr int shell_b(int s) {
    constexpr int t[3] = {0, 0, 1};
    return t[s];
  }
  __host__ __device__ static constexpr int shell_first(int s) {
    constexpr int t[3] = {0, 1, 5};
    return t[s];
  }
  __host__ __device__ static constexpr int shell_size(int s) {
    constexpr int t[3] = {1, 4, 4};
    return t[s];
  }
};

template <class S>
__host__ __device__ constexpr int e2_of(int i) {
  return S::ex(i) * S::ex(i) + S::ey(i) * S::ey(i);
}
template <class S>
__host__ __device__ constexpr int shell_of(int i) {
  int s = 0;
  for (int k = 0; k < S::NSHELL; ++k)
    if (i >= S::shell_first(k)) s = k;
  return s;
}

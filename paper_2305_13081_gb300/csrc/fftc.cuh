// Stockham FFT with the transform length known at compile time.
//
// The same algorithm, pass order and twiddle table as fft_lines (radix 9
// passes, then one radix 3, for powers of three; radix 8 passes, then one
// radix 4 or 2, for powers of two), but every divisor, stride and offset is
// a constant: line and butterfly indices come from multiply-shifts, the
// loads and stores of a butterfly use immediate offsets from one base
// address, and the pass loop is unrolled. The runtime version spends most of
// its issue slots on integer index arithmetic; this one spends them on the
// butterflies. Two layouts:
//   rows    (COL = false): line l, element i at buf[l N + i] (x lines);
//   columns (COL = true):  line c, element i at buf[i CW + c] (a strip of
//                          CW columns, all CW lines present).
#pragma once

#include "fftmech_dev.cuh"

namespace fftmech {

__host__ __device__ constexpr int pow_of(int n, int p) { return n % p == 0 ? 1 + pow_of(n / p, p) : 0; }

// Radix of pass s of a length-n plan (the order of factor_plan).
__host__ __device__ constexpr int radix_at(int n, int s) {
  const int c3 = pow_of(n, 3), c2 = pow_of(n, 2);
  const int n9 = c3 / 2, n3 = c3 % 2, n8 = c2 / 3, r2 = c2 % 3;
  return s < n9 ? 9 : s < n9 + n3 ? 3 : s < n9 + n3 + n8 ? 8 : s == n9 + n3 + n8 ? (r2 == 2 ? 4 : r2 == 1 ? 2 : 1) : 1;
}

// Lengths with a compile-time plan: 2^a or 3^b (mixed lengths use fft_lines).
__host__ __device__ constexpr bool fixed_len_ok(int n) {
  int m = n;
  while (m % 3 == 0) m /= 3;
  int k = n;
  while (k % 2 == 0) k /= 2;
  return n >= 2 && (m == 1 || k == 1);
}

// One pass: radix R, sub-transform length NS before the pass, nlines lines
// (rows) or CW lines (columns). Each thread takes butterflies tid + b bd,
// b < BM: PassBatch<R> for rows; for columns with THR > 0 (the block has
// exactly THR threads) as many as the pass needs. All loads precede the
// barrier, all stores follow it.
// No post-processing of a pass's outputs.
struct NoPost {
  template <typename T>
  __device__ __forceinline__ void operator()(cx<T>&, int, int) const {}
};

template <typename T, int S, int N, int R, int NS, bool COL, int CW, int THR, class Post>
__device__ __forceinline__ void fftc_pass(cx<T>* buf, const cx<T>* __restrict__ tw, int nlines, int tid,
                                          Post& post) {
  constexpr int BM = (COL && THR > 0) ? ((N / R) * CW + THR - 1) / THR : PassBatch<R>::value;
  constexpr int NB = N / R;
  const int total = COL ? NB * CW : NB * nlines;
  // the block size as a constant where it is one: the butterfly indices
  // tid + b THR then fold into immediate offsets
  const int bstride = (COL && THR > 0) ? THR : (int)blockDim.x;
  cx<T> v[BM][R];
  int jb[BM];
#pragma unroll
  for (int b = 0; b < BM; ++b) {
    const int idx = tid + b * bstride;
    if (idx < total) {
      int in;
      if constexpr (COL) {
        in = idx;  // (j, c) at j CW + c: element j of column c
        jb[b] = idx;
      } else {
        const int line = idx / NB, j = idx - line * NB;
        in = line * N + j;
        jb[b] = in;
      }
#pragma unroll
      for (int t = 0; t < R; ++t) v[b][t] = buf[in + t * NB * (COL ? CW : 1)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BM; ++b) {
    const int idx = tid + b * bstride;
    if (idx < total) {
      int j, base0;
      if constexpr (COL) {
        j = jb[b] / CW;
        base0 = jb[b] - j * CW;  // the column
      } else {
        const int line = jb[b] / N;
        j = jb[b] - line * N;
        base0 = line * N;
      }
      const int q = j / NS, k = j - q * NS;
      if constexpr (NS > 1) {
        const cx<T>* w = tw + k * (R - 1);
#pragma unroll
        for (int t = 1; t < R; ++t) {
          const cx<T> wt = w[t - 1];
          v[b][t] = (S < 0) ? cmul(v[b][t], wt) : cmulc(v[b][t], wt);
        }
      }
      dft<T, R, S>(v[b]);
      if constexpr (NS * R == N) {  // the last pass: outputs are final (frequency q NS R + k + t NS)
#pragma unroll
        for (int t = 0; t < R; ++t) post(v[b][t], q * NS * R + k + t * NS, base0);
      }
      const int out = (q * NS * R + k) * (COL ? CW : 1) + base0;
#pragma unroll
      for (int t = 0; t < R; ++t) buf[out + t * NS * (COL ? CW : 1)] = v[b][t];
    }
  }
  __syncthreads();
}

template <typename T, int S, int N, int P, int NS, bool COL, int CW, int THR, class Post>
__device__ __forceinline__ void fftc_from(cx<T>* buf, const cx<T>* tw, int nlines, int tid, Post& post) {
  if constexpr (NS < N) {
    constexpr int R = radix_at(N, P);
    static_assert(R > 1 && N % (NS * R) == 0, "plan mismatch");
    fftc_pass<T, S, N, R, NS, COL, CW, THR>(buf, tw, nlines, tid, post);
    fftc_from<T, S, N, P + 1, NS * R, COL, CW, THR>(buf, tw + NS * (R - 1), nlines, tid, post);
  }
}

// Full transform of nlines rows (COL = false) or of a CW-column strip
// (COL = true) in place; tw: the plan's twiddles (any memory space).
// Requires, for every pass, lines * N / r <= PassBatch<r> * blockDim.x, or
// for columns with THR > 0 a block of exactly THR threads.
// post(value, frequency, line) is applied to every output of the last pass
// before it is stored (for columns, line = the column in the strip).
template <typename T, int S, int N, bool COL, int CW = 1, int THR = 0, class Post = NoPost>
__device__ __forceinline__ void fftc(cx<T>* buf, const cx<T>* tw, int nlines, Post&& post = Post()) {
  static_assert(fixed_len_ok(N), "compile-time plans cover 2^a and 3^b");
  // opaque copies of the table pointer and the thread index: keep the
  // compiler from hoisting every pass's index arithmetic and twiddle loads
  // out of a caller's loop into (spilled) registers
  const cx<T>* twl = tw;
  int tid = threadIdx.x;
  asm volatile("" : "+l"(twl), "+r"(tid));
  fftc_from<T, S, N, 0, 1, COL, CW, THR>(buf, twl, nlines, tid, post);
}

}  // namespace fftmech

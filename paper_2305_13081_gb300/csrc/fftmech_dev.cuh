// Device building blocks: complex arithmetic, small DFT butterflies, the
// mixed-radix (2, 3, 4, 8, 9) Stockham autosort FFT on lines held in shared
// memory, and deterministic FP64 block reductions.
//
// The Stockham pass used here: with sub-transform length Ns before the pass
// and radix r, butterfly j (0 <= j < n/r) reads x[j + t n/r] (t < r),
// multiplies input t by w_{Ns r}^{t (j mod Ns)}, takes a radix-r DFT and
// writes output t to (j div Ns) Ns r + (j mod Ns) + t Ns. Passes run in place
// in shared memory: every thread loads all of its butterflies' inputs into
// registers, the block synchronises, then every thread writes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fftmech {

// Programmatic dependent launch: wait until the kernel launched before this
// one on the stream has completed and its writes are visible, then allow the
// next kernel of the stream to begin launching (its blocks take free SM slots
// and run up to their own wait). A kernel launched with the programmatic
// stream-serialisation attribute must call this in every block before it
// reads or writes anything another kernel writes or reads, and before it can
// return; under a plain launch both instructions return at once.
__device__ __forceinline__ void grid_dep_sync() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename T>
struct __align__(2 * sizeof(T)) cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> c; c.re = a; c.im = b; return c; }
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return mk(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
template <typename T>
__device__ __forceinline__ cx<T> scal(cx<T> a, T s) { return mk(a.re * s, a.im * s); }
// multiply by s*i for s = +1 / -1
template <typename T, int S>
__device__ __forceinline__ cx<T> muli(cx<T> a) { return S > 0 ? mk(-a.im, a.re) : mk(a.im, -a.re); }

// ---------------------------------------------------------------- butterflies
// S = -1: forward exp(-2 pi i / r); S = +1: inverse.
template <typename T, int S>
__device__ __forceinline__ void dft2(cx<T>* v) {
  cx<T> a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}

template <typename T, int S>
__device__ __forceinline__ void dft3(cx<T>& a, cx<T>& b, cx<T>& c) {
  const T h3 = T(0.8660254037844386);  // sin(2 pi / 3)
  cx<T> t1 = b + c;
  cx<T> t2 = a - scal(t1, T(0.5));
  cx<T> t3 = scal(b - c, T(S) * h3);  // times i below
  a = a + t1;
  b = t2 + muli<T, 1>(t3);
  c = t2 - muli<T, 1>(t3);
}

template <typename T, int S>
__device__ __forceinline__ void dft4(cx<T>& a, cx<T>& b, cx<T>& c, cx<T>& d) {
  cx<T> s0 = a + c, s1 = a - c, s2 = b + d, s3 = muli<T, S>(b - d);
  a = s0 + s2;
  c = s0 - s2;
  b = s1 + s3;
  d = s1 - s3;
}

template <typename T, int S>
__device__ __forceinline__ void dft8(cx<T>* v) {
  const T r2 = T(0.7071067811865476);
  cx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  cx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<T, S>(e0, e1, e2, e3);
  dft4<T, S>(o0, o1, o2, o3);
  // w8^m = exp(S i 2 pi m / 8)
  cx<T> w1 = mk(r2, T(S) * r2);
  cx<T> w3 = mk(-r2, T(S) * r2);
  o1 = cmul(o1, w1);
  o2 = muli<T, S>(o2);
  o3 = cmul(o3, w3);
  v[0] = e0 + o0; v[4] = e0 - o0;
  v[1] = e1 + o1; v[5] = e1 - o1;
  v[2] = e2 + o2; v[6] = e2 - o2;
  v[3] = e3 + o3; v[7] = e3 - o3;
}

template <typename T, int S>
__device__ __forceinline__ void dft9(cx<T>* v) {
  // 9 = 3 x 3: inner DFT3 over n1 for each n2 (x[3 n1 + n2]), twiddle
  // w9^(n2 k1), outer DFT3 over n2 for each k1; output X[k1 + 3 k2].
  const T c1 = T(0.766044443118978), s1 = T(0.6427876096865393);    // 2 pi / 9
  const T c2 = T(0.17364817766693041), s2 = T(0.984807753012208);   // 4 pi / 9
  const T c4 = T(-0.9396926207859083), s4 = T(0.3420201433256689);  // 8 pi / 9
  cx<T> a0 = v[0], a1 = v[3], a2 = v[6];
  cx<T> b0 = v[1], b1 = v[4], b2 = v[7];
  cx<T> d0 = v[2], d1 = v[5], d2 = v[8];
  dft3<T, S>(a0, a1, a2);
  dft3<T, S>(b0, b1, b2);
  dft3<T, S>(d0, d1, d2);
  b1 = cmul(b1, mk(c1, T(S) * s1));
  b2 = cmul(b2, mk(c2, T(S) * s2));
  d1 = cmul(d1, mk(c2, T(S) * s2));
  d2 = cmul(d2, mk(c4, T(S) * s4));
  dft3<T, S>(a0, b0, d0);
  dft3<T, S>(a1, b1, d1);
  dft3<T, S>(a2, b2, d2);
  v[0] = a0; v[3] = b0; v[6] = d0;
  v[1] = a1; v[4] = b1; v[7] = d1;
  v[2] = a2; v[5] = b2; v[8] = d2;
}

template <typename T, int R, int S>
__device__ __forceinline__ void dft(cx<T>* v) {
  if constexpr (R == 2) dft2<T, S>(v);
  else if constexpr (R == 3) dft3<T, S>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<T, S>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<T, S>(v);
  else dft9<T, S>(v);
}

// ---------------------------------------------------------------- index helpers
// Division by a block-invariant divisor 1 <= d < 2^16 for 0 <= x < 2^16:
// q = floor(x * m / 2^32) with m = ceil(2^32 / d). Writing m = 2^32/d + e
// (0 <= e < 1), x m / 2^32 = x/d + x e / 2^32 < x/d + 2^-16, while the
// fractional part of x/d is at most 1 - 1/d <= 1 - 2^-16, so the floor is
// exact. Integer-only (one multiply-high per division).
struct FastDiv {
  unsigned int m;
  int d;
  __host__ __device__ static unsigned int magic(int d_) { return d_ > 1 ? 0xFFFFFFFFu / (unsigned)d_ + 1u : 0u; }
  __device__ __forceinline__ explicit FastDiv(int d_) : m(magic(d_)), d(d_) {}
  // from a multiplier computed elsewhere (no division in the kernel)
  __device__ __forceinline__ FastDiv(unsigned int m_, int d_) : m(m_), d(d_) {}
  __device__ __forceinline__ int div(int x) const { return d > 1 ? (int)__umulhi((unsigned)x, m) : x; }
};

// ---------------------------------------------------------------- double-float
// (hi, lo) += a * p for a = ah + al (a double split into two floats), p a
// float: the product's rounding error comes from one FMA (Dekker), the sum's
// from TwoSum (Knuth), and the result is renormalised (FastTwoSum).
__device__ __forceinline__ void df_axpy(float& hi, float& lo, float ah, float al, float p) {
  const float prod = ah * p;
  const float perr = fmaf(ah, p, -prod);
  const float dlo = fmaf(al, p, perr);
  const float s = hi + prod;
  const float bb = s - hi;
  float e = (hi - (s - bb)) + (prod - bb);
  e += lo + dlo;
  const float h2 = s + e;
  lo = e - (h2 - s);
  hi = h2;
}

// ---------------------------------------------------------------- staged copies
// Contiguous global -> shared copy with U loads in flight per thread.
template <int U, typename E>
__device__ __forceinline__ void g2s(E* __restrict__ dst, const E* __restrict__ src, int n) {
  const int bd = blockDim.x;
  for (int i = threadIdx.x; i < n; i += U * bd) {
    E v[U];
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (i + k * bd < n) v[k] = src[i + k * bd];
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (i + k * bd < n) dst[i + k * bd] = v[k];
  }
}

// Contiguous global -> shared copy with 16-byte vector loads (U in flight
// per thread): a misaligned head and the tail are copied element by element.
// RO: the source is not written during the kernel (read-only data path).
template <int U, bool RO, typename E>
__device__ __forceinline__ void g2s_vec(E* __restrict__ dst, const E* __restrict__ src, int n) {
  constexpr int PER = 16 / (int)sizeof(E);
  if constexpr (PER <= 1) {
    g2s<U>(dst, src, n);
  } else {
    const int mis = (int)((reinterpret_cast<uintptr_t>(src) / sizeof(E)) % PER);
    const int head = min(n, (PER - mis) % PER);
    const int nv = (n - head) / PER;
    const int bd = blockDim.x;
    for (int i = threadIdx.x; i < head; i += bd) dst[i] = src[i];
    const int tail0 = head + nv * PER;
    for (int i = tail0 + threadIdx.x; i < n; i += bd) dst[i] = src[i];
    const int4* s4 = reinterpret_cast<const int4*>(src + head);
    E* d = dst + head;
    for (int i = threadIdx.x; i < nv; i += U * bd) {
      int4 v[U];
#pragma unroll
      for (int k = 0; k < U; ++k)
        if (i + k * bd < nv) v[k] = RO ? __ldg(s4 + i + k * bd) : s4[i + k * bd];
#pragma unroll
      for (int k = 0; k < U; ++k)
        if (i + k * bd < nv) {
          const E* e = reinterpret_cast<const E*>(&v[k]);
#pragma unroll
          for (int j = 0; j < PER; ++j) d[(i + k * bd) * PER + j] = e[j];
        }
    }
  }
}

// Rows ys .. ys + W - 1 (periodic in ny) of a [ny][nx] field into dst[W][nx].
template <int U, typename E>
__device__ __forceinline__ void g2s_rows(E* dst, const E* __restrict__ src, int ys, int W, int nx,
                                         int ny) {
  int y = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
  int done = 0;
  while (done < W) {
    const int run = min(W - done, ny - y);
    g2s_vec<U, true>(dst + (size_t)done * nx, src + (size_t)y * nx, run * nx);
    done += run;
    y = 0;
  }
}

// Contiguous global -> shared copy with asynchronous copies (cp.async, no
// registers held while the data is in flight): element i of src to dst[i].
// E of 4, 8 or 16 bytes, both arrays aligned to sizeof(E). The copies
// complete at g2s_async_wait(); a __syncthreads() after it makes them
// visible to the whole block.
template <typename E>
__device__ __forceinline__ void g2s_async(E* dst, const E* src, int n) {
  static_assert(sizeof(E) == 4 || sizeof(E) == 8 || sizeof(E) == 16, "cp.async copies 4, 8 or 16 bytes");
  const unsigned base = (unsigned)__cvta_generic_to_shared(dst);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned d = base + (unsigned)(i * (int)sizeof(E));
    const E* s = src + i;
    if constexpr (sizeof(E) == 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(s) : "memory");
    else if constexpr (sizeof(E) == 8)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(s) : "memory");
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(s) : "memory");
  }
}
__device__ __forceinline__ void g2s_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Contiguous shared -> global copy.
template <typename E>
__device__ __forceinline__ void s2g(E* __restrict__ dst, const E* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// u[i] += a * p[i] for a double iterate in global memory and a direction in
// shared memory, U read-modify-writes in flight per thread.
template <int U, typename T>
__device__ __forceinline__ void axpy_g(double* __restrict__ u, const T* __restrict__ p, double a, int n) {
  const int bd = blockDim.x;
  for (int i = threadIdx.x; i < n; i += U * bd) {
    double v[U];
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (i + k * bd < n) v[k] = u[i + k * bd];
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (i + k * bd < n) u[i + k * bd] = v[k] + a * (double)p[i + k * bd];
  }
}

// (uh, ul)[i] += a * p[i] in double-float, U updates in flight per thread.
template <int U>
__device__ __forceinline__ void df_axpy_g(float* __restrict__ uh, float* __restrict__ ul,
                                          const float* __restrict__ p, float ah, float al, int n) {
  const int bd = blockDim.x;
  for (int i = threadIdx.x; i < n; i += U * bd) {
    float h[U], l[U];
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (i + k * bd < n) { h[k] = uh[i + k * bd]; l[k] = ul[i + k * bd]; }
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (i + k * bd < n) {
        df_axpy(h[k], l[k], ah, al, p[i + k * bd]);
        uh[i + k * bd] = h[k];
        ul[i + k * bd] = l[k];
      }
  }
}

// ---------------------------------------------------------------- plans
constexpr int kMaxPass = 12;

// One 1D transform length, factored into passes. The radix of pass s is the
// 4-bit field s of `rcode`; the twiddles of pass s start after those of the
// earlier passes (sum of Ns (r - 1)): entry k (r - 1) + t - 1 =
// exp(-2 pi i k t / (Ns r)).
template <typename T>
struct FftPlanDev {
  int n;
  int npass;
  unsigned long long rcode;
  const cx<T>* tw;
  // FastDiv multipliers of pass s: mag[s] for Ns (sub-transform length
  // before the pass), mag[kMaxPass + s] for n / r (butterflies per line).
  // They follow the twiddles in the plan's buffer (at byte offset
  // tw_smem_twiddles(n)); kernels copy both to shared memory and point mag
  // there (NULL: computed in place).
  const unsigned int* mag;
};

// Butterflies a thread keeps in registers per pass: about nine points for
// every radix, so one launch shape serves all passes.
template <int R>
struct PassBatch {
  static constexpr int value = R >= 8 ? 1 : (R == 4 ? 2 : (R == 3 ? 3 : 4));
};

// Element (line, i) of a batch of lines sits at buf[line * ls + i * is].
// lines_fast: consecutive threads take consecutive lines (column batches
// stored [i][line]); otherwise consecutive butterflies of one line.
template <typename T, int R, int S>
__device__ __forceinline__ void stockham_pass(cx<T>* buf, int n, int Ns, const cx<T>* __restrict__ tw,
                                              int nlines, int ls, int is, bool lines_fast, const FastDiv& dlines,
                                              unsigned int mnb, const FastDiv& dn) {
  constexpr int BM = PassBatch<R>::value;
  const int nb = n / R;
  const int total = nb * nlines;
  const FastDiv dl = lines_fast ? dlines : FastDiv(mnb, nb);
  cx<T> v[BM][R];
  int lj[BM];
#pragma unroll
  for (int b = 0; b < BM; ++b) {
    const int idx = threadIdx.x + b * blockDim.x;
    if (idx < total) {
      int line, j;
      if (lines_fast) { j = dl.div(idx); line = idx - j * nlines; }
      else { line = dl.div(idx); j = idx - line * nb; }
      lj[b] = line * 65536 + j;
      const cx<T>* src = buf + (size_t)line * ls;
#pragma unroll
      for (int t = 0; t < R; ++t) v[b][t] = src[(j + t * nb) * is];
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BM; ++b) {
    const int idx = threadIdx.x + b * blockDim.x;
    if (idx < total) {
      const int line = lj[b] >> 16, j = lj[b] & 0xFFFF;
      const int q = dn.div(j);
      const int k = j - q * Ns;
      if (Ns > 1) {
        const cx<T>* w = tw + k * (R - 1);
#pragma unroll
        for (int t = 1; t < R; ++t) {
          const cx<T> wt = w[t - 1];
          v[b][t] = (S < 0) ? cmul(v[b][t], wt) : cmulc(v[b][t], wt);
        }
      }
      dft<T, R, S>(v[b]);
      cx<T>* dst = buf + (size_t)line * ls;
      const int base = q * Ns * R + k;
#pragma unroll
      for (int t = 0; t < R; ++t) dst[(base + t * Ns) * is] = v[b][t];
    }
  }
  __syncthreads();
}

// Radix families: a kernel is compiled for the radices its transform
// lengths use, which keeps register pressure at that of the largest
// butterfly instead of the sum over all five.
enum RadixFamily { FAM_9 = 1, FAM_93 = 2, FAM_842 = 3, FAM_ALL = 4 };

template <int FAM, int R>
struct FamilyHas {
  static constexpr bool value =
      FAM == FAM_ALL || (FAM == FAM_9 && R == 9) || (FAM == FAM_93 && (R == 9 || R == 3)) ||
      (FAM == FAM_842 && (R == 8 || R == 4 || R == 2));
};

// Full transform of `nlines` lines in place. Requires, for every pass,
// nlines * n / r <= PassBatch<r> * blockDim.x (checked by the host), and
// every radix of the plan in family FAM.
template <typename T, int S, int FAM>
__device__ void fft_lines(cx<T>* buf, const FftPlanDev<T>& p, int nlines, int ls, int is,
                          bool lines_fast) {
  int Ns = 1;
  int off = 0;
  const int n = p.n;
  const unsigned long long code = p.rcode;
  const FastDiv dlines(nlines);  // the only division of the transform
  for (int s = 0; s < p.npass; ++s) {
    const int r = (int)((code >> (4 * s)) & 15ull);
    const cx<T>* tw = p.tw + off;
    const FastDiv dn(p.mag ? p.mag[s] : FastDiv::magic(Ns), Ns);
    const unsigned int mnb = p.mag ? p.mag[kMaxPass + s] : FastDiv::magic(n / r);
    if constexpr (FamilyHas<FAM, 9>::value) {
      if (r == 9) stockham_pass<T, 9, S>(buf, n, Ns, tw, nlines, ls, is, lines_fast, dlines, mnb, dn);
    }
    if constexpr (FamilyHas<FAM, 8>::value) {
      if (r == 8) stockham_pass<T, 8, S>(buf, n, Ns, tw, nlines, ls, is, lines_fast, dlines, mnb, dn);
    }
    if constexpr (FamilyHas<FAM, 4>::value) {
      if (r == 4) stockham_pass<T, 4, S>(buf, n, Ns, tw, nlines, ls, is, lines_fast, dlines, mnb, dn);
    }
    if constexpr (FamilyHas<FAM, 3>::value) {
      if (r == 3) stockham_pass<T, 3, S>(buf, n, Ns, tw, nlines, ls, is, lines_fast, dlines, mnb, dn);
    }
    if constexpr (FamilyHas<FAM, 2>::value) {
      if (r == 2) stockham_pass<T, 2, S>(buf, n, Ns, tw, nlines, ls, is, lines_fast, dlines, mnb, dn);
    }
    off += Ns * (r - 1);
    Ns *= r;
  }
}

// Twiddles of a plan in shared memory: kernels copy the n - 1 entries to
// the start of their dynamic shared memory (with the other staged loads,
// before their first barrier) so the passes read them with short latency.
template <typename T>
__host__ __device__ constexpr size_t tw_smem_twiddles(int n) {
  return ((size_t)(n > 1 ? n - 1 : 0) * sizeof(cx<T>) + 15) & ~size_t(15);
}
template <typename T>
__host__ __device__ constexpr size_t tw_smem_bytes(int n) {
  return tw_smem_twiddles<T>(n) + 2 * kMaxPass * sizeof(unsigned int);
}
template <typename T>
__device__ __forceinline__ FftPlanDev<T> plan_to_smem(const FftPlanDev<T>& p, cx<T>* dst) {
  // twiddles, padding and multipliers: one contiguous 16-byte multiple
  g2s_vec<4, true>(reinterpret_cast<int4*>(dst), reinterpret_cast<const int4*>(p.tw),
                   (int)(tw_smem_bytes<T>(p.n) / sizeof(int4)));
  FftPlanDev<T> q = p;
  q.tw = dst;
  q.mag = reinterpret_cast<const unsigned int*>(reinterpret_cast<const unsigned char*>(dst) +
                                                tw_smem_twiddles<T>(p.n));
  return q;
}

// Host: the multipliers that follow a plan's twiddles (see FftPlanDev).
inline void plan_multipliers(int n, int npass, const int* radix, unsigned int* out) {
  for (int s = 0; s < 2 * kMaxPass; ++s) out[s] = 0u;
  int Ns = 1;
  for (int s = 0; s < npass; ++s) {
    out[s] = FastDiv::magic(Ns);
    out[kMaxPass + s] = FastDiv::magic(n / radix[s]);
    Ns *= radix[s];
  }
}

// fft_lines as a real call: a kernel that keeps much state live across a
// loop around the transform saves it once per call instead of spilling
// inside the butterflies.
template <typename T, int S, int FAM>
__device__ __noinline__ void fft_lines_call(cx<T>* buf, const FftPlanDev<T> p, int nlines, int ls, int is,
                                            bool lines_fast) {
  fft_lines<T, S, FAM>(buf, p, nlines, ls, is, lines_fast);
}

// ---------------------------------------------------------------- reductions
// Linear thread index and thread count of the block (kernels with 2D
// blocks reduce too).
__device__ __forceinline__ int flat_tid() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }
__device__ __forceinline__ int flat_nthreads() { return blockDim.x * blockDim.y * blockDim.z; }
// Sum of K doubles over the block; result valid in thread 0. Uses `scratch`
// (>= 32 * K doubles of shared memory). Deterministic for a fixed launch.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* scratch) {
  const int tid = flat_tid();
  const int lane = tid & 31, wid = tid >> 5;
  const int nw = (flat_nthreads() + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[k * 32 + wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double x = (lane < nw) ? scratch[k * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[k] = x;
    }
  }
  __syncthreads();
}

// Double-float accumulator (h + l, |l| <= ulp(h) / 2): error-free TwoSum
// (Knuth) keeps FP64-like accuracy with float instructions only, which
// float kernels use so that their reductions need no FP64 pipe.
struct dfloat {
  float h, l;
};
__device__ __forceinline__ dfloat df_add(dfloat a, float b) {
  const float s = a.h + b;
  const float bb = s - a.h;
  const float e = (a.h - (s - bb)) + (b - bb);
  const float l = a.l + e;
  const float h2 = s + l;
  return dfloat{h2, l - (h2 - s)};
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float e = (a.h - (s - bb)) + (b.h - bb);
  const float l = a.l + b.l + e;
  const float h2 = s + l;
  return dfloat{h2, l - (h2 - s)};
}
// Numbers of the true residual b - K u (the reliable updates and the
// final check of the mixed path). The FP64 path computes it in double; the
// mixed path in double-float: the pair dfloat (h, l) stands for h + l,
// sums from Knuth's TwoSum, products from an FMA (the
// exact rounding error of h1 h2), renormalised by FastTwoSum; about 2^-48
// relative error per operation on the FP32 pipe, where GB300 runs FP64 at
// a small fraction of that rate. The residual is stored in float, so
// 2^-48 of |b| leaves it accurate to float precision down to |r| ~ 1e-7 |b|
// and to 1e-4 relative at |r| ~ 1e-10 |b|.
__device__ __forceinline__ dfloat df_fast(float s, float e) {
  const float h = s + e;
  return dfloat{h, e - (h - s)};
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float e = ((a.h - (s - bb)) + (b.h - bb)) + (a.l + b.l);
  return df_fast(s, e);
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat{-a.h, -a.l}; }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = a.h * b.h;
  const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)));
  return df_fast(p, e);
}
__device__ __forceinline__ dfloat operator*(dfloat a, float b) {
  const float p = a.h * b;
  const float e = fmaf(a.l, b, fmaf(a.h, b, -p));
  return df_fast(p, e);
}
// The residual's number type for a field type T, and its conversions.
template <typename T>
struct ResidNum {
  using type = double;
};
template <>
struct ResidNum<float> {
  using type = dfloat;
};
template <typename RN>
__device__ __forceinline__ RN rn_c(double x);  // from a double constant
template <>
__device__ __forceinline__ double rn_c<double>(double x) { return x; }
template <>
__device__ __forceinline__ dfloat rn_c<dfloat>(double x) {
  const float h = (float)x;
  return dfloat{h, (float)(x - (double)h)};
}
template <typename RN>
__device__ __forceinline__ RN rn_f(float x);  // from a float (exact)
template <>
__device__ __forceinline__ double rn_f<double>(float x) { return (double)x; }
template <>
__device__ __forceinline__ dfloat rn_f<dfloat>(float x) { return dfloat{x, 0.f}; }
// a value of the field type T (double on the FP64 path, float on the mixed)
template <typename RN, typename T>
__device__ __forceinline__ RN rn_t(T x) {
  if constexpr (sizeof(T) == 4) return rn_f<RN>((float)x);
  else return rn_c<RN>((double)x);
}
// rounded to the field type
__device__ __forceinline__ float rn_out(dfloat a) { return a.h + a.l; }
__device__ __forceinline__ double rn_out(double a) { return a; }

// Block sum of double-float values, returned in thread 0 (others get a
// partial). scratch: 64 floats of shared memory.
__device__ __forceinline__ dfloat block_sum_df2(dfloat v, float* scratch) {
  const int tid = flat_tid();
  const int lane = tid & 31, wid = tid >> 5;
  const int nw = (flat_nthreads() + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const dfloat w{__shfl_down_sync(0xffffffffu, v.h, o), __shfl_down_sync(0xffffffffu, v.l, o)};
    v = df_add(v, w);
  }
  __syncthreads();
  if (lane == 0) {
    scratch[2 * wid] = v.h;
    scratch[2 * wid + 1] = v.l;
  }
  __syncthreads();
  if (wid == 0) {
    v = lane < nw ? dfloat{scratch[2 * lane], scratch[2 * lane + 1]} : dfloat{0.f, 0.f};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const dfloat w{__shfl_down_sync(0xffffffffu, v.h, o), __shfl_down_sync(0xffffffffu, v.l, o)};
      v = df_add(v, w);
    }
  }
  __syncthreads();
  return v;
}
__device__ __forceinline__ double block_sum_df(dfloat v, float* scratch) {
  const dfloat t = block_sum_df2(v, scratch);
  return (double)t.h + (double)t.l;
}

// One ticket of a last-block reduction: an atomic increment with
// acquire-release semantics at GPU scope (it orders the caller's earlier
// partial stores before the increment, and the last block's later loads
// of the other blocks' partials after it).
__device__ __forceinline__ unsigned int ticket_acq_rel(unsigned int* counter) {
  unsigned int prev;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(counter) : "memory");
  return prev;
}

// Publish this block's K partial sums; returns true in every thread of the
// last block to finish, after which partials of all blocks are visible.
template <int K>
__device__ __forceinline__ bool publish_partials(const double (&v)[K], double* partials,
                                                 unsigned int* counter) {
  __shared__ int am_last;
  if (flat_tid() == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)blockIdx.x * K + k] = v[k];
    const unsigned int prev = ticket_acq_rel(counter);
    am_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  return am_last != 0;
}

// v[k] = sum of partials[b K + k] over this thread's blocks b = t, t + bd,
// ... in increasing order (UN loads in flight; the additions keep that
// order, so the result does not depend on the unrolling).
template <int K, int UN = 1>
__device__ __forceinline__ void sum_partials_ordered(double (&v)[K], const double* partials, int total) {
  const int nt = flat_nthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0.0;
  for (int b0 = flat_tid(); b0 < total; b0 += UN * nt) {
    double x[UN][K];
#pragma unroll
    for (int j = 0; j < UN; ++j) {
      const int b = b0 + j * nt;
#pragma unroll
      for (int k = 0; k < K; ++k) x[j][k] = b < total ? __ldcg(partials + (size_t)b * K + k) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < UN; ++j) {
      if (b0 + j * nt < total) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += x[j][k];
      }
    }
  }
}

// In the last block: totals[k] = sum over blocks in index order (thread 0
// returns them; the counter is reset for the next launch). The ticket's
// acquire by thread 0 and the barrier after it order these loads after
// every block's partial stores.
template <int K>
__device__ __forceinline__ void gather_partials(double (&tot)[K], const double* partials,
                                                unsigned int* counter, double* scratch) {
  double v[K];
  sum_partials_ordered<K>(v, partials, (int)gridDim.x);
  block_sum<K>(v, scratch);
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = v[k];
  if (flat_tid() == 0) *counter = 0u;
}

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

}  // namespace fftmech

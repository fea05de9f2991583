// Host-side FFT plans and launch shapes, shared by the context API and the
// allocation-free transform. Nothing here allocates device memory.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>

#include "fftmech_internal.cuh"

namespace fftmech {

struct HostPlan {
  int n = 1;
  int npass = 0;
  int radix[kMaxPass] = {0};
  int twoff[kMaxPass] = {0};
  unsigned long long rcode = 0;
  int rmin = 1;
  int fam = FAM_9;
  cx<float>* tw_f = nullptr;   // device twiddles (owned by whoever filled them)
  cx<double>* tw_d = nullptr;
};

inline bool factor_ok(int n) {
  if (n < 1 || n > 4096) return false;
  int m = n;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

// Factor n = 2^a 3^b into passes: radix 9 and 3 for the powers of three,
// 8, 4, 2 for the powers of two. Sets the radix family of the plan.
inline void factor_plan(int n, HostPlan& p) {
  p = HostPlan();
  p.n = n;
  int m = n, np = 0;
  int rs[kMaxPass];
  while (m % 9 == 0 && np < kMaxPass) { rs[np++] = 9; m /= 9; }
  while (m % 3 == 0 && np < kMaxPass) { rs[np++] = 3; m /= 3; }
  while (m % 8 == 0 && np < kMaxPass) { rs[np++] = 8; m /= 8; }
  while (m % 4 == 0 && np < kMaxPass) { rs[np++] = 4; m /= 4; }
  while (m % 2 == 0 && np < kMaxPass) { rs[np++] = 2; m /= 2; }
  p.npass = np;
  p.rmin = np ? 9 : n;
  int off = 0, Ns = 1;
  bool only9 = true, only93 = true, only842 = true;
  for (int s = 0; s < np; ++s) {
    const int r = rs[s];
    p.radix[s] = r;
    p.twoff[s] = off;
    p.rcode |= (unsigned long long)r << (4 * s);
    p.rmin = std::min(p.rmin, r);
    off += Ns * (r - 1);
    Ns *= r;
    only9 = only9 && r == 9;
    only93 = only93 && (r == 9 || r == 3);
    only842 = only842 && (r == 8 || r == 4 || r == 2);
  }
  p.fam = only9 ? FAM_9 : (only93 ? FAM_93 : (only842 ? FAM_842 : FAM_ALL));
}

// Number of twiddle factors of a plan (n - 1 for n > 1).
inline int twiddle_count(const HostPlan& p) {
  int off = 0, Ns = 1;
  for (int s = 0; s < p.npass; ++s) { off += Ns * (p.radix[s] - 1); Ns *= p.radix[s]; }
  return off;
}

// Twiddles in FP64 on the host: pass s, entry k (r - 1) + t - 1 =
// exp(-2 pi i k t / (Ns r)).
inline void fill_twiddles(const HostPlan& p, cx<double>* out) {
  int Ns = 1, w = 0;
  for (int s = 0; s < p.npass; ++s) {
    const int r = p.radix[s];
    const long long L = (long long)Ns * r;
    for (int k = 0; k < Ns; ++k)
      for (int t = 1; t < r; ++t) {
        const long long kt = ((long long)k * t) % L;
        const double ang = -2.0 * M_PI * (double)kt / (double)L;
        out[w].re = std::cos(ang);
        out[w].im = std::sin(ang);
        ++w;
      }
    Ns *= r;
  }
}

template <typename T>
inline FftPlanDev<T> dev_plan(const HostPlan& p) {
  FftPlanDev<T> d;
  d.n = p.n;
  d.npass = p.npass;
  d.rcode = p.rcode;
  if constexpr (sizeof(T) == 4) d.tw = p.tw_f; else d.tw = p.tw_d;
  d.mag = nullptr;
  return d;
}

inline int round32(int x) { return ((x + 31) / 32) * 32; }

inline int pass_batch(int r) { return r >= 8 ? 1 : (r == 4 ? 2 : (r == 3 ? 3 : 4)); }

// Threads needed so that every pass of `nlines` lines of plan p fits the
// per-thread register batch of the device FFT.
inline int need_threads(const HostPlan& p, int nlines) {
  int need = 1;
  for (int s = 0; s < p.npass; ++s) {
    const int bf = nlines * (p.n / p.radix[s]);
    need = std::max(need, (bf + pass_batch(p.radix[s]) - 1) / pass_batch(p.radix[s]));
  }
  return need;
}

// 2D launch shapes of the residual and column kernels: one row per residual
// block; strips of CW columns (8 for float, 4 for double), halved while the
// batch would have fewer than two strips per SM, within the shared-memory
// budget and the widest column pass fitting 512 threads. Returns false if
// even one row / one column does not fit.
template <typename T>
bool choose_shape(const HostPlan& px, const HostPlan& py, int nsm, size_t optin_total, Shape2& s, int batch = 1) {
  const int nx = px.n, ny = py.n;
  const size_t optin = optin_total - 1024;  // room for the kernels' static shared memory
  const int tmax = 512;
  const size_t budget = std::min<size_t>(optin, sizeof(T) == 4 ? 100 * 1024 : 110 * 1024);
  const size_t twx = tw_smem_bytes<T>(nx), twy = tw_smem_bytes<T>(ny);
  // strip buffer, twiddles and the strip's symbol tables
  auto col_smem = [&](int cw) { return (size_t)ny * cw * sizeof(cx<T>) + twy + (size_t)(ny + cw) * sizeof(T); };
  s = Shape2();
  s.batch = 1;
  s.rows_update = s.rows_dir = 1;  // (row FFT of the bare transform only)
  s.threads_update = s.threads_dir = std::min(tmax, std::max(256, round32(need_threads(px, 1))));
  s.rows_res = 1;
  if (smem_residual<T, 2>(nx, 1) + twx > optin || smem_residual<T, 1>(nx, 1) + twx > optin) return false;
  s.threads_res = std::min(tmax, std::max(256, round32(need_threads(px, 1))));
  int CW = sizeof(T) == 4 ? 8 : 4;
  const bool fixed = sizeof(T) == 4 && (ny == 81 || ny == 243 || ny == 729 || ny == 2187 || ny == 128 ||
                                        ny == 256 || ny == 512 || ny == 1024);
  if (fixed) {
    // compile-time column plans (512 threads, several butterflies each):
    // 64-byte (or 32-byte for 2187) row segments; 4 columns when the batch
    // has fewer than two 8-column strips per SM
    if (ny >= 1024 || (long long)((nx + 7) / 8) * batch < 2LL * nsm) CW = 4;
    if (col_smem(CW) > optin) return false;
    s.cols = CW;
    s.threads_col = 512;
    s.threads_plain = s.threads_update;
    return true;
  }
  // at least two strips per SM (over the batch) when possible
  while (CW > 2 && (long long)((nx + CW - 1) / CW) * batch < 2LL * nsm) CW /= 2;
  while (CW > 1 && (col_smem(CW) > budget || need_threads(py, CW) > tmax)) CW /= 2;
  if (col_smem(CW) > optin || need_threads(py, CW) > tmax) return false;
  s.cols = CW;
  s.threads_col = std::min(tmax, std::max(128, round32(need_threads(py, CW))));
  s.threads_plain = s.threads_update;
  return true;
}

// 3D launch shapes of the FP64 residual bricks (R lines x Zc planes, the
// largest R <= 4 that fits, (R + 2) nx < 2^16 for the kernel's integer
// division, Zc giving about six blocks per SM) and of the y / z line passes
// (strips of CW spectral columns: 16 for float, 8 for double).
template <typename T>
bool choose_shape3(const HostPlan& px, const HostPlan& py, const HostPlan& pz, int nsm, size_t optin_total,
                   int batch, Shape3& s) {
  const int nx = px.n, ny = py.n, nz = pz.n;
  const size_t optin = optin_total - 1024;
  const int tmax = 512;
  const int es = (int)sizeof(T);
  const size_t budget = std::min<size_t>(optin, 110 * 1024);
  s = Shape3();
  s.batch = batch;
  s.nx = nx;
  s.ny = ny;
  s.nz = nz;
  s.sst = (long long)(nx + nx / 2 + 1) * ny * nz;
  const size_t twx = tw_smem_bytes<T>(nx);
  auto res_fits = [&](int r) {
    return (long long)(r + 2) * nx < 65536 && (long long)r * nxs_of(nx, 3) < 65536 &&
           Row3Layout(nx, r, 8, es, 3).total + twx <= optin && Row3Layout(nx, r, 8, es, 1).total + twx <= optin &&
           need_threads(px, 2 * r) <= tmax;
  };
  int rr = std::min(ny, 4);
  while (rr > 1 && !res_fits(rr)) --rr;
  if (!res_fits(rr)) return false;
  s.ry_res = rr;
  {
    const long long nty = (ny + rr - 1) / rr;
    long long nzc = (6LL * nsm + nty * batch - 1) / (nty * batch);
    nzc = std::max(1LL, std::min<long long>(nzc, nz));
    s.zc_res = std::max(std::min(4, nz), (int)((nz + nzc - 1) / nzc));
  }
  s.thr_res = std::min(tmax, std::max(128, round32(need_threads(px, 2 * rr))));
  auto strip = [&](const HostPlan& pl, int& cw, int& thr) {
    int c = sizeof(T) == 4 ? 16 : 8;
    const size_t tw = tw_smem_bytes<T>(pl.n);
    // strip buffer, twiddles and the z pass's symbol tables
    auto bytes = [&](int cc) { return (size_t)pl.n * cc * sizeof(cx<T>) + tw + (size_t)(pl.n + 2 * cc) * sizeof(T); };
    while (c > 1 && (bytes(c) > budget || need_threads(pl, c) > tmax || (long long)pl.n * c >= 65536)) c /= 2;
    if (bytes(c) > optin || need_threads(pl, c) > tmax) return false;
    cw = c;
    thr = std::min(tmax, std::max(128, round32(need_threads(pl, c))));
    return true;
  };
  if (!strip(py, s.cw_y, s.thr_y) || !strip(pz, s.cw_z, s.thr_z)) return false;
  if ((long long)batch > 65535) return false;  // grid.y of the line passes
  return true;
}

// Threads of the fused direction-stencil kernel with L own rows: 512 (its
// element loops and loads gain from every warp; the L + 2 transformed rows
// need at most 512, checked with the shape).
inline int ds_threads(const HostPlan&, int) { return 512; }

// Split iteration: lines per block for the x-line kernels. The largest L
// (at most 16) whose shared memory leaves room for three blocks per SM and
// whose widest FFT pass fits 512 threads, lowered while the launch would
// have fewer than two blocks per SM; the stencil tiles are fixed (64 x 16
// in 2D; 32 x 8 marching through Zc planes in 3D, Zc giving about eight
// blocks per SM).
template <typename T>
bool choose_line_shape(const HostPlan& px, int nlines, int dim, int nxs3, int nsm, size_t optin_total, int batch,
                       LineShape& s) {
  const int nx = px.n;
  const size_t optin = optin_total - 1024;
  const size_t budget = std::min<size_t>(optin, 72 * 1024);
  const int nf = dim == 3 ? 2 : 1;  // D = 3 rows carry two complex fields
  const int Dmax = dim == 3 ? 3 : 2;
  auto ok = [&](int L, bool dir, size_t lim) {
    const size_t sm = dir ? xdir_smem<T>(nx, L, Dmax, dim) : xupd_smem<T>(nx, L, Dmax, dim);
    return sm <= lim && need_threads(px, nf * L) <= 512 && (long long)L * nxs3 < 65536 &&
           (long long)L * nx < 65536;
  };
  auto pick = [&](bool dir) {
    int L = std::min(nlines, 16);
    while (L > 1 && !ok(L, dir, budget)) --L;
    while (L > 1 && (long long)((nlines + L - 1) / L) * batch < 2LL * nsm) --L;
    return ok(L, dir, optin) ? L : 0;
  };
  s = LineShape();
  s.batch = batch;
  s.L_dir = pick(true);
  s.L_upd = pick(false);
  if (!s.L_dir || !s.L_upd) return false;
  s.thr_dir = std::min(512, std::max(256, round32(need_threads(px, nf * s.L_dir))));
  s.thr_upd = std::min(512, std::max(256, round32(need_threads(px, nf * s.L_upd))));
  // the fused direction-stencil kernel (2D), 512 threads a block, at most
  // two blocks per SM (its registers) and as many as its shared memory
  // allows: the L whose launch takes the fewest waves, each wave costing
  // its blocks' transformed rows (L + 2) plus a fixed latency of about four
  // rows' worth; ties go to the larger L
  s.L_ds = 0;
  s.thr_ds = 0;
  if (dim == 2) {
    auto ok_ds = [&](int L, size_t lim) {
      return L >= 1 && L <= nlines && DsLayout<T, 2>(nx, L).total + tw_smem_bytes<T>(nx) <= lim &&
             need_threads(px, L + 2) <= 512 && (long long)(L + 2) * nx < 65536;
    };
    double best = 1e300;
    for (int L = 1; L <= 16; ++L) {
      if (!ok_ds(L, optin)) continue;
      const size_t sm = DsLayout<T, 2>(nx, L).total + tw_smem_bytes<T>(nx) + 1024;
      const long long per_sm = std::max<long long>(1, std::min<long long>(2, (long long)((optin_total + 1024) / sm)));
      const long long blocks = (long long)((nlines + L - 1) / L) * batch;
      const long long waves = (blocks + per_sm * nsm - 1) / (per_sm * nsm);
      const double cost = (double)waves * (4.0 + L + 2);
      if (cost <= best) {
        best = cost;
        s.L_ds = L;
      }
    }
    if (s.L_ds > 0) s.thr_ds = ds_threads(px, s.L_ds);
  }
  return true;
}

// Whether L own rows per block fit the fused direction-stencil kernel (2D).
template <typename T>
bool ds_shape_ok(const HostPlan& px, int L, int ny, size_t optin_total) {
  const int nx = px.n;
  return L >= 1 && L <= ny && DsLayout<T, 2>(nx, L).total + tw_smem_bytes<T>(nx) <= optin_total - 1024 &&
         need_threads(px, L + 2) <= 512 && (long long)(L + 2) * nx < 65536;
}

// Whether L lines per block fit the x-line direction (dir) or update kernel
// (shared memory within optin, widest pass within 512 threads, index ranges
// within 16 bits), and the threads such a block takes.
template <typename T>
bool line_shape_ok(const HostPlan& px, int L, bool dir, int dim, int nxs3, size_t optin_total) {
  const int nx = px.n;
  const int nf = dim == 3 ? 2 : 1;
  const int Dmax = dim == 3 ? 3 : 2;
  const size_t sm = dir ? xdir_smem<T>(nx, L, Dmax, dim) : xupd_smem<T>(nx, L, Dmax, dim);
  return L >= 1 && sm <= optin_total - 1024 && need_threads(px, nf * L) <= 512 && (long long)L * nxs3 < 65536 &&
         (long long)L * nx < 65536;
}
inline int line_threads(const HostPlan& px, int L, int dim) {
  const int nf = dim == 3 ? 2 : 1;
  return std::min(512, std::max(256, round32(need_threads(px, nf * L))));
}

inline void choose_sten_shape(int nx, int ny, int nz, int dim, int nsm, int batch, StenShape& s) {
  s = StenShape();
  s.batch = batch;
  s.threads = 256;
  s.grid = std::max(1, (8 * nsm + batch - 1) / batch);  // blocks per problem, looping over tiles
  if (dim == 2) {
    // warp strips of 30 columns and 8 rows; 4 rows when that gives fewer
    // than 32 strips per SM (small problems: latency, not bandwidth)
    s.tx = 30;
    s.ty = (long long)((nx + 29) / 30) * ((ny + 7) / 8) * batch >= 32LL * nsm ? 8 : 4;
    s.zc = 1;
    return;
  }
  // warp bricks of 30 columns, 4 rows and zc planes: zc from 2 to 16, as
  // long as the bricks give at least 32 warps per SM
  s.tx = 30;
  s.ty = 4;
  const long long strips = (long long)((nx + 29) / 30) * ((ny + 3) / 4) * batch;
  const long long chunks = (32LL * nsm + strips - 1) / strips;
  const long long zc = (nz + chunks - 1) / chunks;
  s.zc = (int)std::max(1LL, std::min<long long>(std::min<long long>(16, nz), std::max(2LL, zc)));
}

// Launch shapes for the bare transform (row FFT + column FFT only), which
// needs far less shared memory than the solver's row kernels.
template <typename T>
bool choose_shape_fft(const HostPlan& px, const HostPlan& py, int nsm, size_t optin_total, Shape2& s) {
  const int nx = px.n, ny = py.n;
  const int tmax = 512;
  const size_t optin = optin_total - 1024;
  int R = std::max(1, std::min(ny, ny / (2 * nsm)));
  auto fits = [&](int r) {
    return (size_t)r * nx * sizeof(cx<T>) + tw_smem_bytes<T>(nx) <= optin && need_threads(px, r) <= tmax;
  };
  while (R > 1 && !fits(R)) --R;
  if (!fits(R)) return false;
  s.batch = 1;
  s.rows_update = s.rows_dir = R;
  s.threads_update = s.threads_dir = s.threads_plain =
      std::min(tmax, std::max(128, round32(need_threads(px, R))));
  s.rows_res = 1;
  s.threads_res = s.threads_update;
  int CW = sizeof(T) == 4 ? 8 : 4;
  while (CW > 2 && (nx + CW - 1) / CW < 2 * nsm) CW /= 2;
  const size_t twy = tw_smem_bytes<T>(ny);
  auto col_smem = [&](int cw) { return (size_t)ny * cw * sizeof(cx<T>) + twy + (size_t)(ny + cw) * sizeof(T); };
  while (CW > 1 && (col_smem(CW) > optin || need_threads(py, CW) > tmax)) CW /= 2;
  if (col_smem(CW) > optin || need_threads(py, CW) > tmax) return false;
  s.cols = CW;
  s.threads_col = std::min(tmax, std::max(128, round32(need_threads(py, CW))));
  return true;
}

}  // namespace fftmech

// z pass of the 3D equilibrium PCG with the reference-medium preconditioner
// (the Moulinec-Suquet reference medium, Sec. 1): z = K0^-1 r per Fourier
// mode, K0 the Galerkin operator grad+^T C0 grad+ of a homogeneous isotropic
// medium (lambda0 = rho mu0, mu0 = 1). With a = D h (forward-difference
// symbol, Sec. 2.6) the mode matrix is the Hermitian 3 x 3
//   K0(k) = |a|^2 I + rho conj(a) a^T + a conj(a)^T
// and z(k) = K0(k)^-1 r(k) / m1 (0 at k = 0), the scale of the Laplace
// multiplier 1 / (m1 |D|^2 h^2).
//
// After the x and y passes a row of the spectrum holds, per (kz, ky), the
// packed pair P = F(r_x + i r_y) over all kx and the half spectrum H =
// F(r_z) over kx = 0 .. nx / 2. A mode's three components need P at k and
// at -k = (nx - kx, ny - ky, nz - kz):
//   R_x(k) = (P(k) + conj(P(-k))) / 2,  R_y(k) = (P(k) - conj(P(-k))) / (2 i),
// R_z(k) = H(k) for kx <= nx / 2, conj(H(-k)) otherwise; the result goes
// back as P'(k) = z_x + i z_y, P'(-k) = conj(z_x) + i conj(z_y), H'(k) = z_z.
// A block therefore takes the pair of line sets ky and ny - ky (A and B)
// and a strip of CW columns kx <= nx / 2: for each line set the packed
// columns kx and nx - kx and the half column kx, six slots of CW columns
// along z. Per (kx, kz) a thread solves two modes:
//   family 1: k = (kx, ky, kz)        from P_A(kx), P_B(nx - kx), H_A(kx);
//   family 2: (kx, ny - ky, nz - kz)  from P_B(kx), P_A(nx - kx), H_B(kx),
// and every P and H value of the six slots is written by exactly one of
// them. Where a column or a line set is its own mirror (kx = 0, 2 kx = nx;
// ky = 0, 2 ky = ny) the duplicate slots are transformed but not stored.
// The Parseval sum <r, M^-1 r> counts each mode once: a solve counts once
// for each of its two modes that the block stores. Partials, the last-block
// ticket and the finalisation follow the Laplace z pass.
#include "kernels3d.cuh"

namespace fftmech {

template <typename T>
__device__ __forceinline__ T re_dot(cx<T> a, cx<T> b) { return a.re * b.re + a.im * b.im; }  // Re(conj(a) b)

// z = K0(a)^-1 r * f (f = 1 / m1), K0 = s I + rho conj(a) a^T + a conj(a)^T
// by its adjugate; returns 0 at a = 0.
template <typename T>
__device__ __forceinline__ void ms_solve3(const cx<T> (&a)[3], T rho, T f, const cx<T> (&r)[3], cx<T> (&z)[3]) {
  const T l0 = a[0].re * a[0].re + a[0].im * a[0].im;
  const T l1 = a[1].re * a[1].re + a[1].im * a[1].im;
  const T l2 = a[2].re * a[2].re + a[2].im * a[2].im;
  const T s = l0 + l1 + l2;
  if (!(s > T(0))) {
    z[0] = z[1] = z[2] = mk(T(0), T(0));
    return;
  }
  // K_ij = s d_ij + rho conj(a_i) a_j + a_i conj(a_j): diagonal s + (rho + 1) |a_i|^2,
  // off-diagonal (i < j) with w = conj(a_i) a_j: rho w + conj(w)
  auto off = [&](int i, int j) {
    const T wre = a[i].re * a[j].re + a[i].im * a[j].im, wim = a[i].re * a[j].im - a[i].im * a[j].re;
    return mk((rho + T(1)) * wre, (rho - T(1)) * wim);
  };
  const T d0 = s + (rho + T(1)) * l0, d1 = s + (rho + T(1)) * l1, d2 = s + (rho + T(1)) * l2;
  const cx<T> b = off(0, 1), c = off(0, 2), e = off(1, 2);
  auto cj = [](cx<T> x) { return mk(x.re, -x.im); };
  auto mul = [](cx<T> x, cx<T> y) { return mk(x.re * y.re - x.im * y.im, x.re * y.im + x.im * y.re); };
  auto nrm = [](cx<T> x) { return x.re * x.re + x.im * x.im; };
  // adjugate of [[d0, b, c], [b*, d1, e], [c*, e*, d2]]
  const T A00 = d1 * d2 - nrm(e), A11 = d0 * d2 - nrm(c), A22 = d0 * d1 - nrm(b);
  const cx<T> ce = mul(c, cj(e)), be = mul(b, e), cbs = mul(cj(b), c);
  const cx<T> A01 = mk(ce.re - b.re * d2, ce.im - b.im * d2);   // c e* - b d2
  const cx<T> A02 = mk(be.re - c.re * d1, be.im - c.im * d1);   // b e - c d1
  const cx<T> A12 = mk(cbs.re - e.re * d0, cbs.im - e.im * d0); // b* c - d0 e
  // the matrix is Hermitian, so is its adjugate: A10 = conj(A01), ...
  const cx<T> A10 = cj(A01), A20 = cj(A02), A21 = cj(A12);
  // det = row 0 of K times column 0 of adj(K) (real)
  const T det = d0 * A00 + mul(b, A10).re + mul(c, A20).re;
  T g;
  if constexpr (sizeof(T) == 4) g = __fdividef(f, det);
  else g = f / det;
  const cx<T> z0 = mk(A00 * r[0].re, A00 * r[0].im) + mul(A01, r[1]) + mul(A02, r[2]);
  const cx<T> z1 = mul(A10, r[0]) + mk(A11 * r[1].re, A11 * r[1].im) + mul(A12, r[2]);
  const cx<T> z2 = mul(A20, r[0]) + mul(A21, r[1]) + mk(A22 * r[2].re, A22 * r[2].im);
  z[0] = scal(z0, g);
  z[1] = scal(z1, g);
  z[2] = scal(z2, g);
}

// The six slots of a block's strip: packed column kx, packed mirror nx - kx
// and half column kx of line set A, then the same of line set B.
enum { MS_PA = 0, MS_PAM = 1, MS_HA = 2, MS_PB = 3, MS_PBM = 4, MS_HB = 5, MS_SLOTS = 6 };

// NL > 0: a compile-time plan of NL points along z and strips of CWC
// columns (float, kLineThreads threads); NL = 0: the runtime plan of family FL.
template <typename T, int FL, int NL, int CWC>
__global__ void FFTMECH_BOUNDS3 k3_zpass_ms(cx<T>* S, long long sst, int nx, int ny, int nz, int nxs,
                                            FftPlanDev<T> pz, Spec<T> sp, int CW, int mode, double* partials,
                                            SolverScalars* sc, int* pmode) {
  const int bp = blockIdx.y;
  extern __shared__ __align__(16) unsigned char smem_all[];
  unsigned char* smem = smem_all + tw_smem_bytes<T>(pz.n);
  const FftPlanDev<T> pz_s = plan_to_smem(pz, reinterpret_cast<cx<T>*>(smem_all));
  if constexpr (NL > 0) {
    nz = NL;
    CW = CWC;
  }
  const int ncs = MS_SLOTS * CW;
  cx<T>* Bf = reinterpret_cast<cx<T>*>(smem);        // [kz][slot]
  cx<T>* AZ = Bf + (size_t)nz * ncs;                 // a_z per line frequency
  cx<T>* AX = AZ + nz;                               // a_x of the strip's columns
  const int H = nx / 2 + 1;
  const int nstrips = (H + CW - 1) / CW;
  const int kyA = blockIdx.x / nstrips, strip = blockIdx.x - kyA * nstrips;
  const int kyB = kyA == 0 ? 0 : ny - kyA;
  const int x0 = strip * CW, nc = min(CW, H - x0);
  for (int i = threadIdx.x; i < nz; i += blockDim.x) AZ[i] = sp.az[i];
  if ((int)threadIdx.x < CW) AX[threadIdx.x] = (int)threadIdx.x < nc ? sp.ax[x0 + threadIdx.x] : mk(T(0), T(0));
  grid_dep_sync();  // plan and tables are constant; everything below follows the previous kernel
  sc += bp;
  if (pmode) pmode += bp;
  if (!col_active(mode, pmode, sc)) return;
  if (mode == COL_ITER && pmode && *pmode == 1) mode = COL_TRUE;  // reliable update of this problem
  const bool store = mode != COL_NORM && mode != COL_TRUENORM;
  const cx<T> ayA = sp.ay[kyA], ayB = sp.ay[kyB];
  const bool self_line = kyA == kyB;
  cx<T>* Sb = S + (size_t)bp * sst;
  const size_t lstride = (size_t)ny * nxs;  // between consecutive z of one column
  auto gcol = [&](int slot, int kx) {       // column of a slot in its row
    const int g = slot % 3;
    return g == 0 ? kx : (g == 1 ? (kx == 0 ? 0 : nx - kx) : nx + kx);
  };
  const int n = nz * ncs;
  const FastDiv dn(ncs), dcw(CW);
  for (int i = threadIdx.x; i < n; i += 8 * blockDim.x) {
    cx<T> t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int ii = i + k * blockDim.x;
      if (ii < n) {
        const int z = dn.div(ii), sl = ii - z * ncs;
        const int slot = dcw.div(sl), c = sl - slot * CW;
        const int ky = slot < 3 ? kyA : kyB;
        t[k] = c < nc ? Sb[(size_t)z * lstride + (size_t)ky * nxs + gcol(slot, x0 + c)] : mk(T(0), T(0));
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (i + k * (int)blockDim.x < n) Bf[i + k * blockDim.x] = t[k];
  }
  __syncthreads();
  if constexpr (NL > 0) fftc<T, -1, NL, true, MS_SLOTS * CWC, kLineThreads>(Bf, pz_s.tw, MS_SLOTS * CWC);
  else fft_lines<T, -1, FL>(Bf, pz_s, ncs, 1, ncs, true);
  __syncthreads();
  const T m1 = sp.m1b ? (T)sp.m1b[bp] : sp.m1_t;
  const T rho = sp.rho_t;
  const T finv = T(1) / m1;
  const T invN = sp.invN_t;
  Acc<T> acc;
  T part = T(0);
  int cnt = 0;
  auto at = [&](int z, int slot, int c) -> cx<T>& { return Bf[(size_t)z * ncs + slot * CW + c]; };
  auto unpack = [](cx<T> pk, cx<T> pm, cx<T>& rx, cx<T>& ry) {  // pm = P(-k)
    rx = mk(T(0.5) * (pk.re + pm.re), T(0.5) * (pk.im - pm.im));
    ry = mk(T(0.5) * (pk.im + pm.im), T(-0.5) * (pk.re - pm.re));
  };
  for (int i = threadIdx.x; i < nz * nc; i += blockDim.x) {
    const int kz = i / nc, c = i - kz * nc;
    const int kzn = kz == 0 ? 0 : nz - kz;
    const int kx = x0 + c;
    const bool self_col = kx == 0 || 2 * kx == nx;
    // family 1: k = (kx, kyA, kz), -k in slot PBM at kzn
    cx<T> r1[3], z1[3], r2[3], z2[3];
    unpack(at(kz, MS_PA, c), at(kzn, MS_PBM, c), r1[0], r1[1]);
    r1[2] = at(kz, MS_HA, c);
    const cx<T> a1[3] = {AX[c], ayA, AZ[kz]};
    ms_solve3<T>(a1, rho, finv, r1, z1);
    // family 2: (kx, kyB, kzn), its mirror (nx - kx, kyA, kz) in slot PAM at kz
    unpack(at(kzn, MS_PB, c), at(kz, MS_PAM, c), r2[0], r2[1]);
    r2[2] = at(kzn, MS_HB, c);
    const cx<T> a2[3] = {AX[c], ayB, AZ[kzn]};
    ms_solve3<T>(a2, rho, finv, r2, z2);
    // Parseval: each solve once per stored mode of its pair
    const T w1 = T(1) + ((self_col || self_line) ? T(0) : T(1));
    const T w2 = (self_line ? T(0) : T(1)) + (self_col ? T(0) : T(1));
    part += w1 * (re_dot(r1[0], z1[0]) + re_dot(r1[1], z1[1]) + re_dot(r1[2], z1[2])) +
            w2 * (re_dot(r2[0], z2[0]) + re_dot(r2[1], z2[1]) + re_dot(r2[2], z2[2]));
    if (++cnt == 8) {  // non-negative terms
      acc.add(part);
      part = T(0);
      cnt = 0;
    }
    if (store) {
      for (int q = 0; q < 3; ++q) {
        z1[q] = scal(z1[q], invN);
        z2[q] = scal(z2[q], invN);
      }
      at(kz, MS_PA, c) = mk(z1[0].re - z1[1].im, z1[0].im + z1[1].re);
      at(kzn, MS_PBM, c) = mk(z1[0].re + z1[1].im, z1[1].re - z1[0].im);
      at(kz, MS_HA, c) = z1[2];
      at(kzn, MS_PB, c) = mk(z2[0].re - z2[1].im, z2[0].im + z2[1].re);
      at(kz, MS_PAM, c) = mk(z2[0].re + z2[1].im, z2[1].re - z2[0].im);
      at(kzn, MS_HB, c) = z2[2];
    }
  }
  acc.add(part);
  if (store) {
    __syncthreads();
    if constexpr (NL > 0) fftc<T, 1, NL, true, MS_SLOTS * CWC, kLineThreads>(Bf, pz_s.tw, MS_SLOTS * CWC);
    else fft_lines<T, 1, FL>(Bf, pz_s, ncs, 1, ncs, true);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int z = dn.div(i), sl = i - z * ncs;
      const int slot = dcw.div(sl), c = sl - slot * CW;
      if (c >= nc) continue;
      const int kx = x0 + c;
      const bool self_col = kx == 0 || 2 * kx == nx;
      if (slot >= 3 && self_line) continue;               // line set B is line set A
      if ((slot == MS_PAM || slot == MS_PBM) && self_col) continue;  // the mirror column is the column
      const int ky = slot < 3 ? kyA : kyB;
      Sb[(size_t)z * lstride + (size_t)ky * nxs + gcol(slot, kx)] = Bf[i];
    }
  }
  __shared__ double red[32];
  __shared__ float redf[64];
  const double bt[1] = {acc.block_total(redf, red)};
  double* part_b = partials + (size_t)bp * gridDim.x;
  if (publish_partials<1>(bt, part_b, &sc->cnt[1])) {
    double tot[1];
    gather_partials<1>(tot, part_b, &sc->cnt[1], red);
    if (threadIdx.x == 0) finalize_col(sc, mode, tot[0] * sp.invN, pmode);
  }
}

// Blocks per problem: (ny / 2 + 1) line-set pairs x strips of CW of the
// nx / 2 + 1 columns.
int zpass_ms_blocks(int nx, int ny, int CW) { return (ny / 2 + 1) * ((nx / 2 + 1 + CW - 1) / CW); }

size_t zpass_ms_smem(int nz, int CW, int es_complex, size_t tw) {
  return (size_t)nz * MS_SLOTS * CW * es_complex + (size_t)(nz + CW) * es_complex + tw;
}

template <typename T, int FL, int NL, int CWC>
cudaError_t launch3_zpass_ms(cx<T>* S, long long sst, int nx, int ny, int nz, int nxs, const FftPlanDev<T>& pz,
                             const Spec<T>& sp, int CW, int threads, int batch, int mode, double* partials,
                             SolverScalars* sc, int* pmode, cudaStream_t st) {
  const size_t sm = zpass_ms_smem(nz, CW, (int)sizeof(cx<T>), tw_smem_bytes<T>(nz));
  static SmemOptIn cfg;
  cudaError_t e = opt_in_smem(k3_zpass_ms<T, FL, NL, CWC>, sm, cfg);
  if (e != cudaSuccess) return e;
  const dim3 grid(zpass_ms_blocks(nx, ny, CW), batch > 0 ? batch : 1);
  return launch_dep(k3_zpass_ms<T, FL, NL, CWC>, grid, dim3(NL > 0 ? kLineThreads : threads), sm, st, S, sst, nx,
                    ny, nz, nxs, pz, sp, CW, mode, partials, sc, pmode);
}

template <typename T>
cudaError_t launch3_zpass_ms_f(int fz, cx<T>* S, long long sst, int nx, int ny, int nz, int nxs,
                               const FftPlanDev<T>& pz, const Spec<T>& sp, int CW, int threads, int batch, int mode,
                               double* partials, SolverScalars* sc, int* pmode, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    // compile-time plans for the benchmark lengths at the strip width the
    // host picks for them (six slots of CW columns within 512 threads)
    if (nz == 81 && CW == 4)
      return launch3_zpass_ms<T, FAM_ALL, 81, 4>(S, sst, nx, ny, nz, nxs, pz, sp, CW, threads, batch, mode, partials,
                                                  sc, pmode, st);
    if (nz == 243 && CW == 2)
      return launch3_zpass_ms<T, FAM_ALL, 243, 2>(S, sst, nx, ny, nz, nxs, pz, sp, CW, threads, batch, mode,
                                                   partials, sc, pmode, st);
    if (nz == 729 && CW == 1)
      return launch3_zpass_ms<T, FAM_ALL, 729, 1>(S, sst, nx, ny, nz, nxs, pz, sp, CW, threads, batch, mode,
                                                   partials, sc, pmode, st);
  }
#define FFTMECH_C(F) \
  launch3_zpass_ms<T, F, 0, 0>(S, sst, nx, ny, nz, nxs, pz, sp, CW, threads, batch, mode, partials, sc, pmode, st)
  FFTMECH_FAMILY_SWITCH(fz, FFTMECH_C)
#undef FFTMECH_C
}

template cudaError_t launch3_zpass_ms_f<float>(int, cx<float>*, long long, int, int, int, int,
                                               const FftPlanDev<float>&, const Spec<float>&, int, int, int, int,
                                               double*, SolverScalars*, int*, cudaStream_t);
template cudaError_t launch3_zpass_ms_f<double>(int, cx<double>*, long long, int, int, int, int,
                                                const FftPlanDev<double>&, const Spec<double>&, int, int, int, int,
                                                double*, SolverScalars*, int*, cudaStream_t);

}  // namespace fftmech

// Homogenised RVE diffusion (Eqs. diffusion, diffusion-final, phi-fft) with
// a choice of gradient operator (Sec. 2.6: forward difference, central
// difference, 8th-order central difference, Fourier i xi), for the
// operator comparison of Fig. 2. The operator is applied in Fourier space
// with its symbol D(k), so every variant runs the same kernels:
//   K phi = D^H F[kappa(x) F^-1(D phi_hat)],  f = -D^H F[kappa(x) G],
// PCG on the spectral vector phi_hat with the preconditioner 1 / |D|^2 (0
// where D vanishes). Per iteration one inverse and one forward transform of
// the gradient (two real components packed as g_x + i g_y, the third in a
// second field in 3D). FP64 throughout: the comparison is about the
// discretisation, not the arithmetic.
//   k_var_grad: W1 = (D_x + i D_y) P (component-wise: D_x P + i D_y P),
//               W2 = D_z P;
//   k_var_flux: W <- kappa(x) (W / N + G) (after the inverse transform);
//   k_var_div:  Q = s sum_a conj(D_a) J_a with J_x, J_y unpacked from
//               Z1 = F(j_x + i j_y) via Z1(-k), J_z = Z2 (after the forward
//               transform);
//   k_var_dot:  block partials of Re sum conj(a) b (summed by the host in
//               a fixed order);
//   k_var_axpy, k_var_precond, k_var_dir: the PCG vector updates.
#include "fftmech_internal.cuh"

namespace fftmech {

static constexpr int kVarThreads = 256;
using cxd = cx<double>;

__device__ __forceinline__ void var_idx(const VarGrid& g, long long i, int& x, int& y, int& z) {
  x = (int)(i % g.nx);
  const long long r = i / g.nx;
  y = (int)(r % g.ny);
  z = (int)(r / g.ny);
}

__device__ __forceinline__ cxd cmuld(cxd a, cxd b) { return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
__device__ __forceinline__ cxd conjd(cxd a) { return mk(a.re, -a.im); }

__global__ void k_var_grad(VarGrid g, const cxd* __restrict__ P, cxd* __restrict__ W1, cxd* __restrict__ W2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    var_idx(g, i, x, y, z);
    const cxd p = P[i];
    const cxd gx = cmuld(g.dx[x], p);
    const cxd gy = g.dim >= 2 ? cmuld(g.dy[y], p) : mk(0.0, 0.0);
    W1[i] = mk(gx.re - gy.im, gx.im + gy.re);  // gx + i gy
    if (g.dim == 3) W2[i] = cmuld(g.dz[z], p);
  }
}

// W1 = g_x + i g_y, W2 = g_z + i (garbage): kappa (g / N + G).
__global__ void k_var_flux(VarGrid g, const uint8_t* __restrict__ phase, double kp, double ks, double G0, double G1,
                           double G2, double invN, cxd* __restrict__ W1, cxd* __restrict__ W2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    const double k = phase[i] ? ks : kp;
    const cxd w = W1[i];
    W1[i] = mk(k * (w.re * invN + G0), k * (w.im * invN + G1));
    if (g.dim == 3) W2[i] = mk(k * (W2[i].re * invN + G2), 0.0);
  }
}

__global__ void k_var_div(VarGrid g, const cxd* __restrict__ Z1, const cxd* __restrict__ Z2, double s,
                          cxd* __restrict__ Q) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    var_idx(g, i, x, y, z);
    const int xm = x == 0 ? 0 : g.nx - x, ym = y == 0 ? 0 : g.ny - y, zm = z == 0 ? 0 : g.nz - z;
    const long long im = ((long long)zm * g.ny + ym) * g.nx + xm;
    const cxd a = Z1[i], b = conjd(Z1[im]);
    const cxd Jx = mk(0.5 * (a.re + b.re), 0.5 * (a.im + b.im));
    const cxd Jy = mk(0.5 * (a.im - b.im), -0.5 * (a.re - b.re));  // (a - b) / (2 i)
    cxd q = cmuld(conjd(g.dx[x]), Jx);
    if (g.dim >= 2) {
      const cxd t = cmuld(conjd(g.dy[y]), Jy);
      q = mk(q.re + t.re, q.im + t.im);
    }
    if (g.dim == 3) {
      const cxd t = cmuld(conjd(g.dz[z]), Z2[i]);
      q = mk(q.re + t.re, q.im + t.im);
    }
    Q[i] = mk(s * q.re, s * q.im);
  }
}

// partials[block] = Re sum conj(a) b over the block's grid-stride share.
__global__ void __launch_bounds__(kVarThreads) k_var_dot(long long n, const cxd* __restrict__ a,
                                                         const cxd* __restrict__ b, double* partials) {
  __shared__ double red[kVarThreads / 32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += a[i].re * b[i].re + a[i].im * b[i].im;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kVarThreads / 32; ++w) t += red[w];
    partials[blockIdx.x] = t;
  }
}

// partials[2 block + 0 / 1] = sum of Re / Im of w over the block's share.
__global__ void __launch_bounds__(kVarThreads) k_var_sum(long long n, const cxd* __restrict__ w, double* partials) {
  __shared__ double red[2][kVarThreads / 32];
  double a = 0.0, b = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    a += w[i].re;
    b += w[i].im;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int k = 0; k < kVarThreads / 32; ++k) {
      ta += red[0][k];
      tb += red[1][k];
    }
    partials[2 * blockIdx.x] = ta;
    partials[2 * blockIdx.x + 1] = tb;
  }
}

// x += alpha p; r -= alpha q
__global__ void k_var_axpy(long long n, double alpha, const cxd* __restrict__ p, const cxd* __restrict__ q,
                           cxd* __restrict__ x, cxd* __restrict__ r) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = mk(x[i].re + alpha * p[i].re, x[i].im + alpha * p[i].im);
    r[i] = mk(r[i].re - alpha * q[i].re, r[i].im - alpha * q[i].im);
  }
}

// z = r / |D|^2 (0 where |D|^2 = 0)
__global__ void k_var_precond(VarGrid g, const cxd* __restrict__ r, cxd* __restrict__ zz) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    var_idx(g, i, x, y, z);
    double d2 = g.dx[x].re * g.dx[x].re + g.dx[x].im * g.dx[x].im;
    if (g.dim >= 2) d2 += g.dy[y].re * g.dy[y].re + g.dy[y].im * g.dy[y].im;
    if (g.dim == 3) d2 += g.dz[z].re * g.dz[z].re + g.dz[z].im * g.dz[z].im;
    const double m = d2 > 0.0 ? 1.0 / d2 : 0.0;
    zz[i] = mk(m * r[i].re, m * r[i].im);
  }
}

// p = z + beta p
__global__ void k_var_dir(long long n, double beta, const cxd* __restrict__ zz, cxd* __restrict__ p) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = mk(zz[i].re + beta * p[i].re, zz[i].im + beta * p[i].im);
}

// out[c N + i] = Re(W_c[i]) / N for the gradient components (W1 = g_x + i g_y, W2 = g_z)
__global__ void k_var_real(VarGrid g, const cxd* __restrict__ W1, const cxd* __restrict__ W2, double scale,
                           double* __restrict__ gx, double* __restrict__ gy, double* __restrict__ gz) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    gx[i] = scale * W1[i].re;
    if (gy) gy[i] = scale * W1[i].im;
    if (gz) gz[i] = scale * W2[i].re;
  }
}

static int var_grid(long long n) {
  long long b = (n + kVarThreads - 1) / kVarThreads;
  return (int)(b < 1 ? 1 : (b > 2048 ? 2048 : b));
}

int var_dot_blocks(long long n) { return var_grid(n); }

cudaError_t launch_var_grad(const VarGrid& g, const cxd* P, cxd* W1, cxd* W2, cudaStream_t st) {
  k_var_grad<<<var_grid(g.N), kVarThreads, 0, st>>>(g, P, W1, W2);
  return cudaGetLastError();
}
cudaError_t launch_var_flux(const VarGrid& g, const uint8_t* phase, double kp, double ks, const double G[3],
                            double invN, cxd* W1, cxd* W2, cudaStream_t st) {
  k_var_flux<<<var_grid(g.N), kVarThreads, 0, st>>>(g, phase, kp, ks, G[0], G[1], G[2], invN, W1, W2);
  return cudaGetLastError();
}
cudaError_t launch_var_div(const VarGrid& g, const cxd* Z1, const cxd* Z2, double s, cxd* Q, cudaStream_t st) {
  k_var_div<<<var_grid(g.N), kVarThreads, 0, st>>>(g, Z1, Z2, s, Q);
  return cudaGetLastError();
}
cudaError_t launch_var_dot(long long n, const cxd* a, const cxd* b, double* partials, cudaStream_t st) {
  k_var_dot<<<var_grid(n), kVarThreads, 0, st>>>(n, a, b, partials);
  return cudaGetLastError();
}
cudaError_t launch_var_sum(long long n, const cxd* w, double* partials, cudaStream_t st) {
  k_var_sum<<<var_grid(n), kVarThreads, 0, st>>>(n, w, partials);
  return cudaGetLastError();
}
cudaError_t launch_var_axpy(long long n, double alpha, const cxd* p, const cxd* q, cxd* x, cxd* r, cudaStream_t st) {
  k_var_axpy<<<var_grid(n), kVarThreads, 0, st>>>(n, alpha, p, q, x, r);
  return cudaGetLastError();
}
cudaError_t launch_var_precond(const VarGrid& g, const cxd* r, cxd* z, cudaStream_t st) {
  k_var_precond<<<var_grid(g.N), kVarThreads, 0, st>>>(g, r, z);
  return cudaGetLastError();
}
cudaError_t launch_var_dir(long long n, double beta, const cxd* z, cxd* p, cudaStream_t st) {
  k_var_dir<<<var_grid(n), kVarThreads, 0, st>>>(n, beta, z, p);
  return cudaGetLastError();
}
cudaError_t launch_var_real(const VarGrid& g, const cxd* W1, const cxd* W2, double scale, double* gx, double* gy,
                            double* gz, cudaStream_t st) {
  k_var_real<<<var_grid(g.N), kVarThreads, 0, st>>>(g, W1, W2, scale, gx, gy, gz);
  return cudaGetLastError();
}

}  // namespace fftmech

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

// ---------------------------------------------------------------- elasticity
// Mechanical equilibrium (Eqs. solid, solid-final) with the same choice of
// gradient operator: K u = D^H F[g C : F^-1(sym D u)], f = -D^H F[g C :
// (E - e I)], PCG on the d spectral displacement components (each N
// numbers) with the preconditioner 1 / |D|^2 per component. The nv tensor
// components of a symmetric field (Voigt order, tensor shears: 2D xx, yy,
// xy; 3D xx, yy, zz, yz, xz, xy) travel as (nv + 1) / 2 complex fields,
// two real components each (v_0 + i v_1, v_2 + i v_3, ...).
struct VarEl {
  int nv, nw;          // Voigt components, packed complex fields
  int a[6], b[6];      // index pair (a, b) of Voigt component v
  cxd* W[3];           // packed fields, N numbers each
};

__device__ __forceinline__ cxd var_sym(const VarGrid& g, const cxd* U, long long i, int x, int y, int z, int a,
                                       int b) {
  auto Dof = [&](int c) { return c == 0 ? g.dx[x] : (c == 1 ? g.dy[y] : g.dz[z]); };
  const cxd ua = U[(long long)a * g.N + i], ub = U[(long long)b * g.N + i];
  if (a == b) return cmuld(Dof(a), ua);
  const cxd s1 = cmuld(Dof(a), ub), s2 = cmuld(Dof(b), ua);
  return mk(0.5 * (s1.re + s2.re), 0.5 * (s1.im + s2.im));
}

// W_w = eps_2w + i eps_(2w+1), eps = sym D u (spectral)
__global__ void k_varel_strain(VarGrid g, VarEl e, const cxd* __restrict__ U) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    var_idx(g, i, x, y, z);
    for (int w = 0; w < e.nw; ++w) {
      const int v0 = 2 * w, v1 = 2 * w + 1;
      const cxd s0 = var_sym(g, U, i, x, y, z, e.a[v0], e.b[v0]);
      const cxd s1 = v1 < e.nv ? var_sym(g, U, i, x, y, z, e.a[v1], e.b[v1]) : mk(0.0, 0.0);
      e.W[w][i] = mk(s0.re - s1.im, s0.im + s1.re);
    }
  }
}

// In real space: eps_v = Re / Im of W (scaled by invN) + E_v; sigma = g (lam
// tr(eps - e I) I + 2 mu (eps - e I)) written back packed. eig, damage:
// NULL = 0; g = (1 - d)^2 + kappa.
__global__ void k_varel_stress(VarGrid g, VarEl e, const uint8_t* __restrict__ phase,
                               const double* __restrict__ eig, const double* __restrict__ damage, double kappa,
                               double lam0, double lam1, double mu0, double mu1, double E0, double E1, double E2,
                               double E3, double E4, double E5, double invN) {
  const double E[6] = {E0, E1, E2, E3, E4, E5};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    double eps[6];
    for (int w = 0; w < e.nw; ++w) {
      const cxd v = e.W[w][i];
      eps[2 * w] = v.re * invN + E[2 * w];
      if (2 * w + 1 < e.nv) eps[2 * w + 1] = v.im * invN + E[2 * w + 1];
    }
    const double ev = eig ? eig[i] : 0.0;
    const int d = g.dim;
    double tr = 0.0;
    for (int c = 0; c < d; ++c) {
      eps[c] -= ev;  // the normal components come first in Voigt order
      tr += eps[c];
    }
    double gg = 1.0;
    if (damage) {
      const double dm = 1.0 - damage[i];
      gg = dm * dm + kappa;
    }
    const bool sol = phase[i] != 0;
    const double lam = gg * (sol ? lam1 : lam0), mu = gg * (sol ? mu1 : mu0);
    double sig[6];
    for (int v = 0; v < e.nv; ++v) sig[v] = 2.0 * mu * eps[v] + (v < d ? lam * tr : 0.0);
    for (int w = 0; w < e.nw; ++w) e.W[w][i] = mk(sig[2 * w], 2 * w + 1 < e.nv ? sig[2 * w + 1] : 0.0);
  }
}

// After the forward transform: sigma_v(k) unpacked from W(k), conj W(-k);
// Q_b = s sum_a conj(D_a) sigma_ab.
__global__ void k_varel_div(VarGrid g, VarEl e, double s, cxd* __restrict__ Q) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    var_idx(g, i, x, y, z);
    const int xm = x == 0 ? 0 : g.nx - x, ym = y == 0 ? 0 : g.ny - y, zm = z == 0 ? 0 : g.nz - z;
    const long long im = ((long long)zm * g.ny + ym) * g.nx + xm;
    cxd sig[6];
    for (int w = 0; w < e.nw; ++w) {
      const cxd a = e.W[w][i], b = conjd(e.W[w][im]);
      sig[2 * w] = mk(0.5 * (a.re + b.re), 0.5 * (a.im + b.im));
      if (2 * w + 1 < e.nv) sig[2 * w + 1] = mk(0.5 * (a.im - b.im), -0.5 * (a.re - b.re));
    }
    const cxd D[3] = {g.dx[x], g.dim >= 2 ? g.dy[y] : mk(0.0, 0.0), g.dim == 3 ? g.dz[z] : mk(0.0, 0.0)};
    cxd q[3] = {mk(0.0, 0.0), mk(0.0, 0.0), mk(0.0, 0.0)};
    for (int v = 0; v < e.nv; ++v) {
      const int a = e.a[v], b = e.b[v];
      const cxd ta = cmuld(conjd(D[a]), sig[v]);
      q[b] = mk(q[b].re + ta.re, q[b].im + ta.im);
      if (a != b) {
        const cxd tb = cmuld(conjd(D[b]), sig[v]);
        q[a] = mk(q[a].re + tb.re, q[a].im + tb.im);
      }
    }
    for (int c = 0; c < g.dim; ++c) Q[(long long)c * g.N + i] = mk(s * q[c].re, s * q[c].im);
  }
}

// x += c
__global__ void k_var_shift(long long n, double c, double* __restrict__ x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += c;
}

// out[v N + i] = Re / Im of the packed fields (scaled)
__global__ void k_varel_real(VarGrid g, VarEl e, double scale, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    for (int w = 0; w < e.nw; ++w) {
      const cxd v = e.W[w][i];
      out[(long long)(2 * w) * g.N + i] = scale * v.re;
      if (2 * w + 1 < e.nv) out[(long long)(2 * w + 1) * g.N + i] = scale * v.im;
    }
  }
}

// ---------------------------------------------------------------- phase field
// AT2 phase field (Eqs. crack, crack-fft) with the same choice of gradient
// operator: K d = (a + H(x)) d + b F^-1(|D|^2 F d), f = H, PCG on the
// spectrum of d with the preconditioner 1 / (m0 + b |D|^2), m0 = a + <H>.
__device__ __forceinline__ double var_d2(const VarGrid& g, int x, int y, int z) {
  double d2 = g.dx[x].re * g.dx[x].re + g.dx[x].im * g.dx[x].im;
  if (g.dim >= 2) d2 += g.dy[y].re * g.dy[y].re + g.dy[y].im * g.dy[y].im;
  if (g.dim == 3) d2 += g.dz[z].re * g.dz[z].re + g.dz[z].im * g.dz[z].im;
  return d2;
}

// W = f (a real field as complex)
__global__ void k_varpf_load(long long n, const double* __restrict__ f, cxd* __restrict__ W) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    W[i] = mk(f[i], 0.0);
}

// W <- (a + H) W / N (after the inverse transform)
__global__ void k_varpf_react(long long n, const double* __restrict__ H, double a, double invN, cxd* __restrict__ W) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double c = (a + H[i]) * invN;
    W[i] = mk(c * W[i].re, c * W[i].im);
  }
}

// Q = W + b |D|^2 P (W: the transformed reaction term); literal: the printed
// Laplacian "i xi . i xi" read as sum D_a^2, Q = W - b (sum D_a^2) P
__global__ void k_varpf_sum(VarGrid g, double b, int literal, const cxd* __restrict__ W, const cxd* __restrict__ P,
                            cxd* __restrict__ Q) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    var_idx(g, i, x, y, z);
    if (literal) {
      cxd s = cmuld(g.dx[x], g.dx[x]);
      if (g.dim >= 2) {
        const cxd t = cmuld(g.dy[y], g.dy[y]);
        s = mk(s.re + t.re, s.im + t.im);
      }
      if (g.dim == 3) {
        const cxd t = cmuld(g.dz[z], g.dz[z]);
        s = mk(s.re + t.re, s.im + t.im);
      }
      const cxd t = cmuld(s, P[i]);
      Q[i] = mk(W[i].re - b * t.re, W[i].im - b * t.im);
    } else {
      const double l = b * var_d2(g, x, y, z);
      Q[i] = mk(W[i].re + l * P[i].re, W[i].im + l * P[i].im);
    }
  }
}

// y = c x (y = x when c = 1), or y += c x
__global__ void k_var_scal(long long n, double c, const cxd* __restrict__ x, cxd* __restrict__ y, int add) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cxd v = mk(c * x[i].re, c * x[i].im);
    y[i] = add ? mk(y[i].re + v.re, y[i].im + v.im) : v;
  }
}

// z = r / (m0 + b |D|^2)
__global__ void k_varpf_precond(VarGrid g, double m0, double b, const cxd* __restrict__ r, cxd* __restrict__ zz) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N; i += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    var_idx(g, i, x, y, z);
    const double m = 1.0 / (m0 + b * var_d2(g, x, y, z));
    zz[i] = mk(m * r[i].re, m * r[i].im);
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

cudaError_t launch_var_shift(long long n, double c, double* x, cudaStream_t st) {
  k_var_shift<<<var_grid(n), kVarThreads, 0, st>>>(n, c, x);
  return cudaGetLastError();
}
VarElSpec var_el_spec(int dim) {
  VarElSpec sp{};
  if (dim == 2) {
    const int a[3] = {0, 1, 0}, b[3] = {0, 1, 1};
    sp.nv = 3;
    for (int v = 0; v < 3; ++v) { sp.a[v] = a[v]; sp.b[v] = b[v]; }
  } else {
    const int a[6] = {0, 1, 2, 1, 0, 0}, b[6] = {0, 1, 2, 2, 2, 1};
    sp.nv = 6;
    for (int v = 0; v < 6; ++v) { sp.a[v] = a[v]; sp.b[v] = b[v]; }
  }
  sp.nw = (sp.nv + 1) / 2;
  return sp;
}
static VarEl var_el(const VarElSpec& sp, cxd* const* W) {
  VarEl e{};
  e.nv = sp.nv;
  e.nw = sp.nw;
  for (int v = 0; v < 6; ++v) { e.a[v] = sp.a[v]; e.b[v] = sp.b[v]; }
  for (int w = 0; w < sp.nw; ++w) e.W[w] = W[w];
  return e;
}
cudaError_t launch_varel_strain(const VarGrid& g, const VarElSpec& sp, cxd* const* W, const cxd* U, cudaStream_t st) {
  k_varel_strain<<<var_grid(g.N), kVarThreads, 0, st>>>(g, var_el(sp, W), U);
  return cudaGetLastError();
}
cudaError_t launch_varel_stress(const VarGrid& g, const VarElSpec& sp, cxd* const* W, const uint8_t* phase,
                                const double* eig, const double* damage, double kappa, const double lam[2],
                                const double mu[2], const double E[6], double invN, cudaStream_t st) {
  k_varel_stress<<<var_grid(g.N), kVarThreads, 0, st>>>(g, var_el(sp, W), phase, eig, damage, kappa, lam[0], lam[1],
                                                         mu[0], mu[1], E[0], E[1], E[2], E[3], E[4], E[5], invN);
  return cudaGetLastError();
}
cudaError_t launch_varel_div(const VarGrid& g, const VarElSpec& sp, cxd* const* W, double s, cxd* Q, cudaStream_t st) {
  k_varel_div<<<var_grid(g.N), kVarThreads, 0, st>>>(g, var_el(sp, W), s, Q);
  return cudaGetLastError();
}
cudaError_t launch_varel_real(const VarGrid& g, const VarElSpec& sp, cxd* const* W, double scale, double* out,
                              cudaStream_t st) {
  k_varel_real<<<var_grid(g.N), kVarThreads, 0, st>>>(g, var_el(sp, W), scale, out);
  return cudaGetLastError();
}

cudaError_t launch_varpf_load(long long n, const double* f, cxd* W, cudaStream_t st) {
  k_varpf_load<<<var_grid(n), kVarThreads, 0, st>>>(n, f, W);
  return cudaGetLastError();
}
cudaError_t launch_varpf_react(long long n, const double* H, double a, double invN, cxd* W, cudaStream_t st) {
  k_varpf_react<<<var_grid(n), kVarThreads, 0, st>>>(n, H, a, invN, W);
  return cudaGetLastError();
}
cudaError_t launch_varpf_sum(const VarGrid& g, double b, int literal, const cxd* W, const cxd* P, cxd* Q,
                             cudaStream_t st) {
  k_varpf_sum<<<var_grid(g.N), kVarThreads, 0, st>>>(g, b, literal, W, P, Q);
  return cudaGetLastError();
}
cudaError_t launch_var_scal(long long n, double c, const cxd* x, cxd* y, int add, cudaStream_t st) {
  k_var_scal<<<var_grid(n), kVarThreads, 0, st>>>(n, c, x, y, add);
  return cudaGetLastError();
}
cudaError_t launch_varpf_precond(const VarGrid& g, double m0, double b, const cxd* r, cxd* z, cudaStream_t st) {
  k_varpf_precond<<<var_grid(g.N), kVarThreads, 0, st>>>(g, m0, b, r, z);
  return cudaGetLastError();
}

}  // namespace fftmech

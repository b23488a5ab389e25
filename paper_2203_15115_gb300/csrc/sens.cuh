// Per-element sensitivity fields from the displacement (Sec. 3.1): strain
// energy s_e = u_e^T (E_e K0) u_e (the element-sensitivity form), Eq. 3.2 at
// the element centroid as printed, and the centroid von Mises stress (the
// measure inside Eq. 3.3's p-norm).  The nodal differences are formed in FP64
// (the Walsh-Hadamard transform of the FP64 displacement), the rest in the
// compute type TC.
#pragma once

#include "afd_common.cuh"

namespace afd {

struct FieldConsts {
  double lam, mu;   // Lame parameters of the unit modulus
  double nu;
  double inv4h;     // 1/(4 h): centroid gradient = linear WHT coefficient / (4 h)
};

template <typename TC>
__device__ __forceinline__ void element_fields(const double (&u)[3][8], TC E, const ElemConsts<TC>& K,
                                               const FieldConsts& F, TC& s_out, TC& tj_out, TC& vm_out) {
  double hd[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int a = 0; a < 8; ++a) hd[c][a] = u[c][a];
    wht8_fwd(hd[c]);
  }
  TC h[3][8], g[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int a = 0; a < 8; ++a) h[c][a] = g[c][a] = (TC)hd[c][a];
  modal_forces(g, E, K);
  TC s = TC(0);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int a = 1; a < 8; ++a) s += h[c][a] * g[c][a];
  s_out = s;
  // centroid strain eps = sym(F), F_dj = h[d][1<<j] / (4h)
  const TC i4h = (TC)F.inv4h;
  const TC exx = h[0][1] * i4h, eyy = h[1][2] * i4h, ezz = h[2][4] * i4h;
  const TC exy = TC(0.5) * (h[0][2] + h[1][1]) * i4h;
  const TC eyz = TC(0.5) * (h[1][4] + h[2][2]) * i4h;
  const TC ezx = TC(0.5) * (h[2][1] + h[0][4]) * i4h;
  const TC tre = exx + eyy + ezz;
  const TC lam = (TC)F.lam * E, mu2 = TC(2) * (TC)F.mu * E;
  const TC sxx = lam * tre + mu2 * exx, syy = lam * tre + mu2 * eyy, szz = lam * tre + mu2 * ezz;
  const TC sxy = mu2 * exy, syz = mu2 * eyz, szx = mu2 * ezx;
  const TC se = sxx * exx + syy * eyy + szz * ezz + TC(2) * (sxy * exy + syz * eyz + szx * ezx);
  const TC trs = sxx + syy + szz;
  const TC nu = (TC)F.nu;
  tj_out = TC(4) / (TC(1) + nu) * se - (TC(1) - TC(3) * nu) / (TC(1) - nu * nu) * trs * tre;
  const TC p = trs / TC(3);
  const TC dxx = sxx - p, dyy = syy - p, dzz = szz - p;
  const TC dd = dxx * dxx + dyy * dyy + dzz * dzz + TC(2) * (sxy * sxy + syz * syz + szx * szx);
  vm_out = sqrt(TC(1.5) * dd);
}

// out[rhs][e] = field `kind` (0 strain energy, 1 Eq. 3.2, 2 von Mises).
template <typename TC>
__global__ void __launch_bounds__(256)
k_element_fields(Grid gr, const double* __restrict__ u, const double* __restrict__ Emod, ElemConsts<TC> K,
                 FieldConsts F, int kind, float* __restrict__ out) {
  const int rhs = blockIdx.y;
  const double* ur = u + (size_t)rhs * gr.vs;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < gr.nelem; e += gridDim.x * blockDim.x) {
    const int i = e % gr.nx, j = (e / gr.nx) % gr.ny, k = e / (gr.nx * gr.ny);
    double uu[3][8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int n = (i + (a & 1)) + gr.nnx * ((j + ((a >> 1) & 1)) + gr.nny * (k + ((a >> 2) & 1)));
#pragma unroll
      for (int c = 0; c < 3; ++c) uu[c][a] = ur[3 * (size_t)n + c];
    }
    TC s, tj, vm;
    element_fields<TC>(uu, (TC)Emod[e], K, F, s, tj, vm);
    out[(size_t)rhs * gr.nelem + e] = (float)(kind == 0 ? s : (kind == 1 ? tj : vm));
  }
}

// Per-block max |x| of a float array per RHS (exact, order independent).
__global__ void __launch_bounds__(256)
k_maxabs_partial(int n, const float* __restrict__ x, float* __restrict__ partials) {
  __shared__ float sh[256];
  const int rhs = blockIdx.y;
  float m = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(x[(size_t)rhs * n + i]));
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[(size_t)rhs * gridDim.x + blockIdx.x] = sh[0];
}

// One block per RHS: max over the partials.
__global__ void k_max_finalize(int nparts, const float* partials, float* out) {
  __shared__ float sh[256];
  const int rhs = blockIdx.x;
  float m = 0.0f;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) m = fmaxf(m, partials[(size_t)rhs * nparts + i]);
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmaxf(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[rhs] = sh[0];
}

// Partial sums of (x / xmax)^p in FP64 per block, per RHS.
__global__ void __launch_bounds__(256)
k_pow_partial(int n, const float* __restrict__ x, const float* __restrict__ xmax, double p, double* partials) {
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  const double m = (double)xmax[rhs];
  double s[1] = {0.0};
  if (m > 0.0) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      s[0] += pow((double)x[(size_t)rhs * n + i] / m, p);
  }
  double o[1];
  block_sum_to_f64<1>(s, red, o);
  if (threadIdx.x == 0) partials[(size_t)rhs * gridDim.x + blockIdx.x] = o[0];
}

// J = f.u partial sums: see k_dot.

// invdiag[n] = 1 / (d0 * sum_{e contains n} E_e): the Jacobi preconditioner,
// from the constant diagonal d0 = h (lam + 4 mu)/9 of the unit element matrix.
template <typename T>
__global__ void k_invdiag(Grid gr, const double* __restrict__ Emod, double d0, T* __restrict__ invdiag) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < gr.nnodes; n += gridDim.x * blockDim.x) {
    const int i = n % gr.nnx, j = (n / gr.nnx) % gr.nny, k = n / (gr.nnx * gr.nny);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int ei = i - (a & 1), ej = j - ((a >> 1) & 1), ek = k - ((a >> 2) & 1);
      if (ei >= 0 && ei < gr.nx && ej >= 0 && ej < gr.ny && ek >= 0 && ek < gr.nz) s += Emod[ei + gr.nx * (ej + gr.ny * ek)];
    }
    invdiag[n] = s > 0.0 ? (T)(1.0 / (d0 * s)) : T(0);
  }
}

}  // namespace afd

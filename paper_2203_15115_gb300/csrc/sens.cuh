// Per-element sensitivity fields from the displacement (Sec. 3.1): strain
// energy s_e = u_e^T (E_e K0) u_e (the element-sensitivity form), Eq. 3.2 at
// the element centroid as printed, and the centroid von Mises stress (the
// measure inside Eq. 3.3's p-norm).  The nodal differences (the
// Walsh-Hadamard transform of the FP64 displacement) are formed in FP64 for
// FP64 fields and in double-float arithmetic for float ones, the rest in the
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
  TC h[3][8], g[3][8];
  if constexpr (sizeof(TC) == 4) {
    // float fields: the transform in double-float arithmetic on the FP32 pipes
    // (the nodal differences to about 2^-44 of u), then rounded to float
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      dfloat hd[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) hd[a] = df_from_double(u[c][a]);
      wht8_fwd(hd);
#pragma unroll
      for (int a = 0; a < 8; ++a) h[c][a] = g[c][a] = (TC)(hd[a].hi + hd[a].lo);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double hd[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) hd[a] = u[c][a];
      wht8_fwd(hd);
#pragma unroll
      for (int a = 0; a < 8; ++a) h[c][a] = g[c][a] = (TC)hd[a];
    }
  }
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

// ---------------------------------------------------------------------------
// Adjoint p-norm stress sensitivity (Eq. 3.3, read with the adjoint state):
//   sigma_PN = (sum_e s_e^p)^(1/p), s_e the centroid von Mises stress,
//   K lambda = -d sigma_PN / d u,
//   T_sigma = 4/(1+nu) sigma(u):eps(lambda) - (1-3 nu)/(1-nu^2) tr sigma(u) tr eps(lambda).
// FP64 throughout (once per topology).
// ---------------------------------------------------------------------------

// Centroid strain (xx, yy, zz, xy, yz, zx; tensor shear) of element (i,j,k)
// from the nodal vector v (stride 3 per node), FP64.
__device__ __forceinline__ void centroid_strain64(const Grid& gr, const double* v, int i, int j, int k, double inv4h,
                                                  double (&eps)[6]) {
  double h[3][8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int n = (i + (a & 1)) + gr.nnx * ((j + ((a >> 1) & 1)) + gr.nny * (k + ((a >> 2) & 1)));
#pragma unroll
    for (int c = 0; c < 3; ++c) h[c][a] = v[3 * (size_t)n + c];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) wht8_fwd(h[c]);
  // centroid gradient F_dj = h[d][1<<j] / (4h)
  eps[0] = h[0][1] * inv4h;
  eps[1] = h[1][2] * inv4h;
  eps[2] = h[2][4] * inv4h;
  eps[3] = 0.5 * (h[0][2] + h[1][1]) * inv4h;
  eps[4] = 0.5 * (h[1][4] + h[2][2]) * inv4h;
  eps[5] = 0.5 * (h[2][1] + h[0][4]) * inv4h;
}

// D[rhs][q][e] (q = xx, yy, zz, xy, yz, zx) = d sigma_PN / d eps_e
//   = 2 mu E_e (3/2) sigma_PN^(1-p) s_e^(p-2) dev(sigma_e)   (dev is traceless)
__global__ void __launch_bounds__(256)
k_pnorm_dsig(Grid gr, const double* __restrict__ u, const double* __restrict__ Emod, FieldConsts F, double p,
             const double* __restrict__ pn, double* __restrict__ D) {
  const int rhs = blockIdx.y;
  const double* ur = u + (size_t)rhs * gr.vs;
  const double PN = pn[rhs];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < gr.nelem; e += gridDim.x * blockDim.x) {
    const int i = e % gr.nx, j = (e / gr.nx) % gr.ny, k = e / (gr.nx * gr.ny);
    double eps[6];
    centroid_strain64(gr, ur, i, j, k, F.inv4h, eps);
    const double E = Emod[e];
    const double tre = eps[0] + eps[1] + eps[2];
    const double lam = F.lam * E, mu2 = 2.0 * F.mu * E;
    double sg[6];
#pragma unroll
    for (int q = 0; q < 3; ++q) sg[q] = lam * tre + mu2 * eps[q];
#pragma unroll
    for (int q = 3; q < 6; ++q) sg[q] = mu2 * eps[q];
    const double pm = (sg[0] + sg[1] + sg[2]) / 3.0;
    double dv[6] = {sg[0] - pm, sg[1] - pm, sg[2] - pm, sg[3], sg[4], sg[5]};
    const double dd = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2] + 2.0 * (dv[3] * dv[3] + dv[4] * dv[4] + dv[5] * dv[5]);
    const double vm = sqrt(1.5 * dd);
    const double coef = (vm > 0.0 && PN > 0.0) ? 1.5 * pow(PN, 1.0 - p) * pow(vm, p - 2.0) : 0.0;
    const double f = mu2 * coef;
    double* Dr = D + (size_t)rhs * 6 * gr.nelem;
#pragma unroll
    for (int q = 0; q < 6; ++q) Dr[(size_t)q * gr.nelem + e] = f * dv[q];
  }
}

// g[rhs][3n+c] = -sum over the elements e of node n of sum_j D_e[c][j] dN_a/dx_j
// at the centroid (dN_a/dx_j = (2 a_j - 1) / (4h)); zero on fixed DOFs.
// Gathered per node in a fixed element order (deterministic).
__global__ void __launch_bounds__(256)
k_pnorm_adjoint_rhs(Grid gr, const double* __restrict__ D, const uint8_t* __restrict__ fixed, double inv4h,
                    double* __restrict__ g) {
  const int rhs = blockIdx.y;
  const double* Dr = D + (size_t)rhs * 6 * gr.nelem;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < gr.nnodes; n += gridDim.x * blockDim.x) {
    const int i = n % gr.nnx, j = (n / gr.nnx) % gr.nny, k = n / (gr.nnx * gr.nny);
    double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      // element (i - bx, j - by, k - bz) holds node n as its local node a = b
      const int ei = i - (b & 1), ej = j - ((b >> 1) & 1), ek = k - ((b >> 2) & 1);
      if (ei < 0 || ei >= gr.nx || ej < 0 || ej >= gr.ny || ek < 0 || ek >= gr.nz) continue;
      const size_t e = (size_t)ei + (size_t)gr.nx * (ej + (size_t)gr.ny * ek);
      const double gx = (2 * (b & 1) - 1) * inv4h, gy = (2 * ((b >> 1) & 1) - 1) * inv4h,
                   gz = (2 * ((b >> 2) & 1) - 1) * inv4h;
      const double xx = Dr[e], yy = Dr[gr.nelem + e], zz = Dr[2 * (size_t)gr.nelem + e];
      const double xy = Dr[3 * (size_t)gr.nelem + e], yz = Dr[4 * (size_t)gr.nelem + e],
                   zx = Dr[5 * (size_t)gr.nelem + e];
      acc[0] += xx * gx + xy * gy + zx * gz;
      acc[1] += xy * gx + yy * gy + yz * gz;
      acc[2] += zx * gx + yz * gy + zz * gz;
    }
    const uint8_t fb = fixed ? fixed[n] : 0;
    double* gr_ = g + (size_t)rhs * gr.vs + 3 * (size_t)n;
#pragma unroll
    for (int c = 0; c < 3; ++c) gr_[c] = ((fb >> c) & 1) ? 0.0 : -acc[c];
  }
}

// out[rhs][e] = T_sigma at the centroid from u and the adjoint lambda.
__global__ void __launch_bounds__(256)
k_stress_topo(Grid gr, const double* __restrict__ u, const double* __restrict__ lam_adj,
              const double* __restrict__ Emod, FieldConsts F, float* __restrict__ out) {
  const int rhs = blockIdx.y;
  const double* ur = u + (size_t)rhs * gr.vs;
  const double* lr = lam_adj + (size_t)rhs * gr.vs;
  const double nu = F.nu;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < gr.nelem; e += gridDim.x * blockDim.x) {
    const int i = e % gr.nx, j = (e / gr.nx) % gr.ny, k = e / (gr.nx * gr.ny);
    double eu[6], el[6];
    centroid_strain64(gr, ur, i, j, k, F.inv4h, eu);
    centroid_strain64(gr, lr, i, j, k, F.inv4h, el);
    const double E = Emod[e];
    const double tre = eu[0] + eu[1] + eu[2];
    const double lam = F.lam * E, mu2 = 2.0 * F.mu * E;
    double sg[6];
#pragma unroll
    for (int q = 0; q < 3; ++q) sg[q] = lam * tre + mu2 * eu[q];
#pragma unroll
    for (int q = 3; q < 6; ++q) sg[q] = mu2 * eu[q];
    const double se = sg[0] * el[0] + sg[1] * el[1] + sg[2] * el[2] + 2.0 * (sg[3] * el[3] + sg[4] * el[4] + sg[5] * el[5]);
    const double trs = sg[0] + sg[1] + sg[2], trl = el[0] + el[1] + el[2];
    out[(size_t)rhs * gr.nelem + e] = (float)(4.0 / (1.0 + nu) * se - (1.0 - 3.0 * nu) / (1.0 - nu * nu) * trs * trl);
  }
}

}  // namespace afd

// Deflated Jacobi-PCG building blocks (Sec. 3.5): fused vector updates with
// partial dot products, the deflation restriction W^T v (force and moment sums
// per node group) and prolongation W y (a rigid motion per group), the coarse
// apply with the explicit inverse of E = W^T K W, and the per-RHS scalar
// recurrences, all on the device so that a chunk of iterations can be
// captured in one CUDA graph.
#pragma once

#include "afd_common.cuh"

namespace afd {

constexpr int RED_BLOCKS = 608;   // 4 x 152 SMs: grid of the vector kernels
constexpr int RED_THREADS = 256;

// Per-RHS scalar state of the (inner) deflated PCG.
struct CGState {
  double rz;        // r.z of the current iterate
  double alpha, beta;
  double rr;        // r.r of the current iterate
  double target2;   // stop when rr <= target2
  int iters;
  int max_iters;
  int done;         // 1: converged or stopped; kernels skip this RHS
  int status;       // 0 ok, AFD_ERR_NOT_CONVERGED, AFD_ERR_NAN
};

// z = r * invdiag (zero on fixed DOFs), partial sums of r.z and r.r
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
k_precond_dot(int ndof, const T* __restrict__ r, const T* __restrict__ invdiag, T* __restrict__ z,
              double* partials, const CGState* st) {
  __shared__ double red[64];
  const int rhs = blockIdx.y;
  if (st && st[rhs].done) return;
  const size_t off = (size_t)rhs * ndof;
  T s[2] = {T(0), T(0)};
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < ndof; d += gridDim.x * blockDim.x) {
    const T rv = r[off + d];
    const T zv = rv * invdiag[d / 3];
    z[off + d] = zv;
    s[0] += rv * zv;
    s[1] += rv * rv;
  }
  double o[2];
  block_sum_to_f64<2>(s, red, o);
  if (threadIdx.x == 0) {
    partials[((size_t)rhs * gridDim.x + blockIdx.x) * 2 + 0] = o[0];
    partials[((size_t)rhs * gridDim.x + blockIdx.x) * 2 + 1] = o[1];
  }
}

// x += alpha p; r -= alpha q; z = r * invdiag; partial sums of r.z, r.r
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
k_cg_update(int ndof, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z, const T* __restrict__ p,
            const T* __restrict__ q, const T* __restrict__ invdiag, double* partials, const CGState* st) {
  __shared__ double red[64];
  const int rhs = blockIdx.y;
  if (st[rhs].done) return;
  const T alpha = (T)st[rhs].alpha;
  const size_t off = (size_t)rhs * ndof;
  T s[2] = {T(0), T(0)};
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < ndof; d += gridDim.x * blockDim.x) {
    const size_t i = off + d;
    x[i] = fma(alpha, p[i], x[i]);
    const T rv = fma(-alpha, q[i], r[i]);
    r[i] = rv;
    const T zv = rv * invdiag[d / 3];
    z[i] = zv;
    s[0] += rv * zv;
    s[1] += rv * rv;
  }
  double o[2];
  block_sum_to_f64<2>(s, red, o);
  if (threadIdx.x == 0) {
    partials[((size_t)rhs * gridDim.x + blockIdx.x) * 2 + 0] = o[0];
    partials[((size_t)rhs * gridDim.x + blockIdx.x) * 2 + 1] = o[1];
  }
}

// Sum nparts partials (stride `stride`, component `comp`) of one RHS in a fixed order.
__device__ inline double sum_partials(const double* p, int nparts, int stride, int comp) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += p[(size_t)i * stride + comp];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  double out = sh[0];
  __syncthreads();
  return out;
}

enum FinMode { FIN_INIT = 0, FIN_ALPHA = 1, FIN_BETA = 2 };

// One block per RHS (256 threads).
//  FIN_ALPHA: alpha = rho / (p.Ap).
//  FIN_INIT / FIN_BETA: rho = r.z + (W^T r).mu (the preconditioned residual
//  y = z + W mu of the two-level operator), r.r, beta = rho_new / rho_old,
//  convergence test on r.r and the iteration cap.
__global__ void k_finalize(int mode, const double* partials, int nparts, CGState* st, int* done_flags,
                           const double* wr, const double* mu, int nc) {
  const int rhs = blockIdx.x;
  CGState& s = st[rhs];
  if (s.done) return;
  const double* p = partials + (size_t)rhs * nparts * (mode == FIN_ALPHA ? 1 : 2);
  if (mode == FIN_ALPHA) {
    const double pap = sum_partials(p, nparts, 1, 0);
    if (threadIdx.x == 0) {
      if (!(pap > 0.0) || !isfinite(pap)) {
        s.status = isfinite(pap) ? -3 : -5;
        s.done = 1;
        if (done_flags) done_flags[rhs] = 1;
      } else {
        s.alpha = s.rz / pap;
      }
    }
    return;
  }
  const double rz = sum_partials(p, nparts, 2, 0);
  const double rr = sum_partials(p, nparts, 2, 1);
  // coarse part of rho, fixed order
  __shared__ double sh[256];
  double c = 0.0;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) c += wr[(size_t)rhs * nc + i] * mu[(size_t)rhs * nc + i];
  sh[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double rho = rz + sh[0];
    if (!isfinite(rr) || !isfinite(rho)) {
      s.status = -5;
      s.done = 1;
    } else {
      if (mode == FIN_BETA) {
        s.beta = rho / s.rz;
        s.iters += 1;
      } else {
        s.beta = 0.0;
      }
      s.rz = rho;
      s.rr = rr;
      if (rr <= s.target2) {
        s.done = 1;
        s.status = 0;
      } else if (s.iters >= s.max_iters) {
        s.done = 1;
        s.status = -3;
      }
    }
    if (done_flags) done_flags[rhs] = s.done;
  }
}

// ---------------------------------------------------------------------------
// Deflation (Sec. 3.5; coarse space = rigid-body modes of agglomerated groups)
// ---------------------------------------------------------------------------

// W^T of one or two vectors (Sec. 3.5 deflation space): for each group G the
// sums over its free DOFs of (v, r x v), r = x_node - c_G, i.e. force and
// moment about the group centroid.  out_a[rhs][6G+q] = (W^T a)_G,
// out_b = W^T b when b is given.  One block per (group, rhs); FP64 output.
template <typename T>
__global__ void __launch_bounds__(256)
k_restrict(Grid gr, Groups gp, const T* __restrict__ a, const T* __restrict__ b, const uint8_t* __restrict__ fixed,
           double* __restrict__ out_a, double* __restrict__ out_b, const CGState* st) {
  __shared__ double red[32 * 12];
  const int G = blockIdx.x, rhs = blockIdx.y;
  if (st && st[rhs].done) return;
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  const int ilo = gp.g * Gx, ihi = (Gx == gp.ngx - 1) ? gr.nx : gp.g * Gx + gp.g - 1;
  const int jlo = gp.g * Gy, jhi = (Gy == gp.ngy - 1) ? gr.ny : gp.g * Gy + gp.g - 1;
  const int klo = gp.g * Gz, khi = (Gz == gp.ngz - 1) ? gr.nz : gp.g * Gz + gp.g - 1;
  const T cx = (T)(0.5 * gp.h * (ilo + ihi)), cy = (T)(0.5 * gp.h * (jlo + jhi)), cz = (T)(0.5 * gp.h * (klo + khi));
  const int lx = ihi - ilo + 1, ly = jhi - jlo + 1, lz = khi - klo + 1;
  const int cnt = lx * ly * lz;
  const size_t off = (size_t)rhs * gr.ndof;
  T s[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) s[q] = T(0);
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int i = ilo + q % lx, j = jlo + (q / lx) % ly, k = klo + q / (lx * ly);
    const int n = i + gr.nnx * (j + gr.nny * k);
    const uint8_t fb = fixed ? fixed[n] : 0;
    const T rx = (T)(gp.h * i) - cx, ry = (T)(gp.h * j) - cy, rz = (T)(gp.h * k) - cz;
#pragma unroll
    for (int which = 0; which < 2; ++which) {
      const T* v = which == 0 ? a : b;
      if (which == 1 && !b) break;
      const T vx = (fb & 1) ? T(0) : v[off + 3 * (size_t)n + 0];
      const T vy = (fb & 2) ? T(0) : v[off + 3 * (size_t)n + 1];
      const T vz = (fb & 4) ? T(0) : v[off + 3 * (size_t)n + 2];
      T* o = s + 6 * which;
      o[0] += vx;
      o[1] += vy;
      o[2] += vz;
      o[3] += ry * vz - rz * vy;
      o[4] += rz * vx - rx * vz;
      o[5] += rx * vy - ry * vx;
    }
  }
  double o[12];
  block_sum_to_f64<12>(s, red, o);
  if (threadIdx.x == 0) {
    const int nc = 6 * gp.ng;
#pragma unroll
    for (int q = 0; q < 6; ++q) out_a[(size_t)rhs * nc + 6 * G + q] = o[q];
    if (b)
#pragma unroll
      for (int q = 0; q < 6; ++q) out_b[(size_t)rhs * nc + 6 * G + q] = o[6 + q];
  }
}

// W mu at node n of group G: t + omega x r (zero on fixed DOFs).
template <typename T>
__device__ __forceinline__ void prolong_node(const Grid& gr, const Groups& gp, const double* mu, int i, int j, int k,
                                             T (&w)[3]) {
  const int Gx = group_of_axis(i, gp.g, gp.ngx), Gy = group_of_axis(j, gp.g, gp.ngy), Gz = group_of_axis(k, gp.g, gp.ngz);
  const int G = Gx + gp.ngx * (Gy + gp.ngy * Gz);
  const double* m = mu + 6 * G;
  const T rx = (T)(gp.h * i - group_centroid_axis(Gx, gp.g, gp.ngx, gr.nnx, gp.h));
  const T ry = (T)(gp.h * j - group_centroid_axis(Gy, gp.g, gp.ngy, gr.nny, gp.h));
  const T rz = (T)(gp.h * k - group_centroid_axis(Gz, gp.g, gp.ngz, gr.nnz, gp.h));
  const T tx = (T)m[0], ty = (T)m[1], tz = (T)m[2], ox = (T)m[3], oy = (T)m[4], oz = (T)m[5];
  w[0] = tx + (oy * rz - oz * ry);
  w[1] = ty + (oz * rx - ox * rz);
  w[2] = tz + (ox * ry - oy * rx);
}

// p = beta p + z + W mu   (mode 0; beta from the state)
// x = W mu                (mode 1)
// x += W mu               (mode 2)
// p = z + W mu            (mode 3)
template <typename T>
__global__ void __launch_bounds__(256)
k_prolong(int mode, Grid gr, Groups gp, T* __restrict__ p, const T* __restrict__ z, const double* __restrict__ mu,
          const uint8_t* __restrict__ fixed, const CGState* st) {
  const int rhs = blockIdx.y;
  if (st && st[rhs].done) return;
  const T beta = (mode == 0 && st) ? (T)st[rhs].beta : T(0);
  const size_t off = (size_t)rhs * gr.ndof;
  const double* m = mu + (size_t)rhs * 6 * gp.ng;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < gr.nnodes; n += gridDim.x * blockDim.x) {
    const int i = n % gr.nnx, j = (n / gr.nnx) % gr.nny, k = n / (gr.nnx * gr.nny);
    T w[3];
    prolong_node(gr, gp, m, i, j, k, w);
    const uint8_t fb = fixed ? fixed[n] : 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t d = off + 3 * (size_t)n + c;
      const T wc = ((fb >> c) & 1) ? T(0) : w[c];
      if (mode == 0) p[d] = fma(beta, p[d], z[d] + wc);
      else if (mode == 1) p[d] = wc;
      else if (mode == 3) p[d] = z[d] + wc;
      else p[d] += wc;
    }
  }
}

// mu[rhs] = Einv (va[rhs] - vb[rhs]) (vb nullable); one warp per row, all RHS
// at once (Einv symmetric, row-major).
__global__ void __launch_bounds__(256)
k_coarse_apply(int nc, int nrhs, const double* __restrict__ Einv, const double* __restrict__ va,
               const double* __restrict__ vb, double* __restrict__ mu, const CGState* st) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nc) return;
  const double* row = Einv + (size_t)warp * nc;
  for (int r = 0; r < nrhs; ++r) {
    if (st && st[r].done) continue;
    const double* ar = va + (size_t)r * nc;
    const double* br = vb ? vb + (size_t)r * nc : nullptr;
    double s = 0.0;
    for (int c = lane; c < nc; c += 32) s = fma(row[c], br ? ar[c] - br[c] : ar[c], s);
    s = warp_sum(s);
    if (lane == 0) mu[(size_t)r * nc + warp] = s;
  }
}

// ---------------------------------------------------------------------------
// Mixed-precision refinement helpers
// ---------------------------------------------------------------------------

// u64 += (double) d32  (per RHS; skip RHS whose outer loop has converged)
__global__ void k_accumulate(int ndof, int nrhs, double* __restrict__ u, const float* __restrict__ d, const int* skip) {
  const int rhs = blockIdx.y;
  if (skip && skip[rhs]) return;
  const size_t off = (size_t)rhs * ndof;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ndof; i += gridDim.x * blockDim.x)
    u[off + i] += (double)d[off + i];
}

template <typename T>
__global__ void k_fill(size_t n, T* __restrict__ x, T v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] = v;
}

// Partial sums of x.y (FP64) per block, per RHS; x, y in type T.
template <typename T, typename U>
__global__ void __launch_bounds__(RED_THREADS)
k_dot(int n, const T* __restrict__ x, const U* __restrict__ y, double* partials) {
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * n;
  double s[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s[0] = fma((double)x[off + i], (double)y[off + i], s[0]);
  double o[1];
  block_sum_to_f64<1>(s, red, o);
  if (threadIdx.x == 0) partials[(size_t)rhs * gridDim.x + blockIdx.x] = o[0];
}

}  // namespace afd

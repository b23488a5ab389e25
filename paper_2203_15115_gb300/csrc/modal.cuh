// Modal analysis (the eigenvalue constraint of Sec. 3.8 and its topological
// sensitivity, Eq. 3.4: K_ff phi = lambda M_ff phi with a lumped mass) and
// linear buckling (Eq. 3.5: (K + lambda K_G) phi = 0) on the deflated solver:
// block LOBPCG for the smallest eigenvalues of a pencil (A, B), with K^-1 by
// the batched solver as the preconditioner.
//
// Mass model (the paper gives none): every node of element e receives
// rho_e h^3 / 8 per direction with rho_e = rho E_e (density follows the
// modulus, so voids add no spurious low-frequency local modes).
#pragma once

#include "afd_common.cuh"
#include "dpcg_kernels.cuh"
#include "sens.cuh"

namespace afd {

constexpr int MODAL_MAX = 36;   // largest Rayleigh-Ritz basis (3 blocks [X, W, P] of up to 12 vectors)

// Lumped mass per DOF (zero on fixed DOFs): m_n = (rho h^3 / 8) sum_{e at n} E_e.
__global__ void k_lumped_mass(Grid gr, const double* __restrict__ Emod, double rho_h3_8,
                              const uint8_t* __restrict__ fixed, double* __restrict__ mass) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < gr.nnodes; n += gridDim.x * blockDim.x) {
    const int i = n % gr.nnx, j = (n / gr.nnx) % gr.nny, k = n / (gr.nnx * gr.nny);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int ei = i - 1 + (a & 1), ej = j - 1 + ((a >> 1) & 1), ek = k - 1 + ((a >> 2) & 1);
      if (ei >= 0 && ei < gr.nx && ej >= 0 && ej < gr.ny && ek >= 0 && ek < gr.nz)
        s += Emod[ei + gr.nx * (ej + gr.ny * ek)];
    }
    const uint8_t fb = fixed ? fixed[n] : 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) mass[3 * (size_t)n + c] = ((fb >> c) & 1) ? 0.0 : rho_h3_8 * s;
  }
}

// SplitMix64 (Steele, Lea and Flood; the constants of Vigna's published
// reference), used as a counter-based generator: one 64-bit output per (seed,
// counter), mapped to a double in [-1, 1).
__device__ __forceinline__ double splitmix_unit(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Starting block: pseudo-random vectors, zero on fixed DOFs (mass zero there).
__global__ void k_modal_start(int ndof, int vs, uint64_t seed, const double* __restrict__ mass, double* __restrict__ X) {
  const int r = blockIdx.y;
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < ndof; d += gridDim.x * blockDim.x)
    X[(size_t)r * vs + d] = mass[d] > 0.0 ? splitmix_unit(seed, (uint64_t)r * ndof + d) : 0.0;
}

// B[r] = M X[r] (diagonal mass).
__global__ void k_mass_apply(int ndof, int vs, const double* __restrict__ mass, const double* __restrict__ X,
                             double* __restrict__ B) {
  const int r = blockIdx.y;
  const size_t off = (size_t)r * vs;
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < ndof; d += gridDim.x * blockDim.x)
    B[off + d] = mass[d] * X[off + d];
}
// Gram matrix partials: parts[b][i kp + j] = sum over this block's DOFs of
// Y[i] Z[j], in a fixed order (tiles of GRAM_T DOFs through shared memory;
// thread t accumulates the pairs t, t + 256, ...).  Reduced by k_gram_final.
constexpr int GRAM_T = 64;
constexpr int GRAM_PAIRS = (MODAL_MAX * MODAL_MAX + 255) / 256;   // pairs per thread
__global__ void __launch_bounds__(256) k_gram(int ndof, int vs, int kp, const double* __restrict__ Y,
                                              const double* __restrict__ Z, double* __restrict__ parts) {
  __shared__ double ys[MODAL_MAX][GRAM_T + 1];
  __shared__ double zs[MODAL_MAX][GRAM_T + 1];
  const int t = threadIdx.x, np = kp * kp;
  double acc[GRAM_PAIRS];
#pragma unroll
  for (int u = 0; u < GRAM_PAIRS; ++u) acc[u] = 0.0;
  for (int base = blockIdx.x * GRAM_T; base < ndof; base += gridDim.x * GRAM_T) {
    for (int q = t; q < kp * GRAM_T; q += blockDim.x) {
      const int r = q / GRAM_T, c = q % GRAM_T, d = base + c;
      ys[r][c] = d < ndof ? Y[(size_t)r * vs + d] : 0.0;
      zs[r][c] = d < ndof ? Z[(size_t)r * vs + d] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < GRAM_PAIRS; ++u) {
      const int pr = t + 256 * u;
      if (pr < np) {
        const int pi = pr / kp, pj = pr % kp;
        double a = acc[u];
        for (int c = 0; c < GRAM_T; ++c) a = fma(ys[pi][c], zs[pj][c], a);
        acc[u] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < GRAM_PAIRS; ++u) {
    const int pr = t + 256 * u;
    if (pr < np) parts[(size_t)blockIdx.x * np + pr] = acc[u];
  }
}
__global__ void k_gram_final(int nparts, int np, const double* __restrict__ parts, double* __restrict__ out) {
  for (int t = threadIdx.x; t < np; t += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += parts[(size_t)b * np + t];
    out[t] = s;
  }
}

// Cyclic Jacobi on a symmetric n x n matrix C (n <= MODAL_MAX) in place,
// run by one warp on shared-memory matrices: every lane takes the same
// rotation (p, q) and applies it to the columns / rows k = lane, lane + 32.
// Eigenvalues end on the diagonal, eigenvectors in the columns of Q.  At most
// 64 sweeps; returns false (in every lane) without convergence.
__device__ bool jacobi_sym(int n, double (&C)[MODAL_MAX][MODAL_MAX], double (&Q)[MODAL_MAX][MODAL_MAX]) {
  const int l = threadIdx.x & 31;
  for (int i = 0; i < n; ++i)
    for (int k = l; k < n; k += 32) Q[i][k] = i == k ? 1.0 : 0.0;
  __syncwarp();
  for (int sweep = 0; sweep < 64; ++sweep) {
    double scale = 0.0;
    for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(C[i][i]));
    bool conv = true;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double cpq = C[p][q];
        if (fabs(cpq) <= 1e-15 * scale) continue;   // the same decision in every lane
        conv = false;
        const double theta = (C[q][q] - C[p][p]) / (2.0 * cpq);
        const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double cs = 1.0 / sqrt(tt * tt + 1.0), sn = tt * cs;
        __syncwarp();   // every lane has read C[p][p], C[p][q], C[q][q]
        for (int k = l; k < n; k += 32) {
          const double a = C[k][p], b = C[k][q];
          C[k][p] = cs * a - sn * b;
          C[k][q] = sn * a + cs * b;
        }
        __syncwarp();
        for (int k = l; k < n; k += 32) {
          const double a = C[p][k], b = C[q][k];
          C[p][k] = cs * a - sn * b;
          C[q][k] = sn * a + cs * b;
        }
        for (int k = l; k < n; k += 32) {
          const double a = Q[k][p], b = Q[k][q];
          Q[k][p] = cs * a - sn * b;
          Q[k][q] = sn * a + cs * b;
        }
        __syncwarp();
      }
    if (conv) return true;
  }
  return false;
}

// Rayleigh-Ritz of A v = theta B v (m x m, row-major) when B may be nearly
// singular (the blocks of LOBPCG grow nearly dependent as it converges): with
// the columns scaled to unit B-norm, B = U diag(d) U^T by Jacobi, the
// directions with d > 1e-12 max d kept, Z = U_keep diag(d_keep)^-1/2,
// C = Z^T A Z by Jacobi, V = Z Q.  The k smallest theta (ascending) and their
// m x k coefficients (row-major, V^T B V = I) are written.  info: 0 ok, 2 no
// convergence, 3 fewer than k directions.  One warp (launch <<<1, 32>>>).
__global__ void __launch_bounds__(32)
k_small_geig_robust(int m, int k, const double* __restrict__ A, const double* __restrict__ Bm,
                    double* __restrict__ lam, double* __restrict__ V, int* info) {
  __shared__ double C[MODAL_MAX][MODAL_MAX], U[MODAL_MAX][MODAL_MAX], Z[MODAL_MAX][MODAL_MAX];
  __shared__ double sc[MODAL_MAX];
  __shared__ int ord[MODAL_MAX];
  const int l = threadIdx.x;
  if (blockIdx.x != 0 || l >= 32) return;
  if (l == 0) *info = 0;
  // columns scaled to unit B-norm first (W and P shrink with the residual; a
  // zero column is dropped), so that the truncation below sees only true
  // dependence, not scale
  for (int i = l; i < m; i += 32) {
    const double d = Bm[i * m + i];
    sc[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
  }
  __syncwarp();
  for (int t = l; t < m * m; t += 32) {
    const int i = t / m, j = t % m;
    C[i][j] = 0.5 * (Bm[i * m + j] + Bm[j * m + i]) * sc[i] * sc[j];
  }
  __syncwarp();
  if (!jacobi_sym(m, C, U)) { if (l == 0) *info = 2; return; }
  double dmax = 0.0;
  for (int i = 0; i < m; ++i) dmax = fmax(dmax, C[i][i]);
  int r = 0;
  for (int j = 0; j < m; ++j) {
    const double d = C[j][j];
    if (!(d > 1e-12 * dmax)) continue;
    const double s = 1.0 / sqrt(d);
    for (int i = l; i < m; i += 32) Z[i][r] = U[i][j] * s;
    ++r;
  }
  if (r < k) { if (l == 0) *info = 3; return; }
  __syncwarp();
  // T = A' Z (m x r, into U) with A' the scaled, symmetrised A; C = Z^T T
  for (int t = l; t < m * r; t += 32) {
    const int i = t / r, b = t % r;
    double s = 0.0;
    for (int j = 0; j < m; ++j) s = fma(0.5 * (A[i * m + j] + A[j * m + i]) * sc[i] * sc[j], Z[j][b], s);
    U[i][b] = s;
  }
  __syncwarp();
  for (int t = l; t < r * r; t += 32) {
    const int a = t / r, b = t % r;
    double s = 0.0;
    for (int i = 0; i < m; ++i) s = fma(Z[i][a], U[i][b], s);
    C[a][b] = s;
  }
  __syncwarp();
  for (int t = l; t < r * r; t += 32) {   // symmetrise (each pair once)
    const int a = t / r, b = t % r;
    if (a < b) {
      const double s = 0.5 * (C[a][b] + C[b][a]);
      C[a][b] = s;
      C[b][a] = s;
    }
  }
  __syncwarp();
  if (!jacobi_sym(r, C, U)) { if (l == 0) *info = 2; return; }
  if (l == 0) {
    for (int i = 0; i < r; ++i) ord[i] = i;
    for (int i = 0; i < r; ++i)
      for (int j = i + 1; j < r; ++j)
        if (C[ord[j]][ord[j]] < C[ord[i]][ord[i]]) {
          const int t = ord[i];
          ord[i] = ord[j];
          ord[j] = t;
        }
    for (int c = 0; c < k; ++c) lam[c] = C[ord[c]][ord[c]];
  }
  __syncwarp();
  for (int t = l; t < m * k; t += 32) {
    const int i = t / k, c = t % k, oc = ord[c];
    double s = 0.0;
    for (int a = 0; a < r; ++a) s = fma(Z[i][a], U[a][oc], s);
    V[i * k + c] = sc[i] * s;
  }
}

// X[r] = sum_j Y[j] V[j][r] for r < kout, Y with kin rows, V kin x kout
// row-major (the Ritz vectors of a block).
__global__ void k_block_combine(int ndof, int vs, int kin, int kout, const double* __restrict__ Y,
                                const double* __restrict__ V, double* __restrict__ X) {
  __shared__ double sv[MODAL_MAX * MODAL_MAX];
  for (int q = threadIdx.x; q < kin * kout; q += blockDim.x) sv[q] = V[q];
  __syncthreads();
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < ndof; d += gridDim.x * blockDim.x) {
    double y[MODAL_MAX];
#pragma unroll
    for (int j = 0; j < MODAL_MAX; ++j) y[j] = j < kin ? Y[(size_t)j * vs + d] : 0.0;
    for (int r = 0; r < kout; ++r) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < MODAL_MAX; ++j)
        if (j < kin) s = fma(y[j], sv[j * kout + r], s);
      X[(size_t)r * vs + d] = s;
    }
  }
}

// R[r] = A X[r] - theta[r] B X[r] (the LOBPCG residual block), zero where
// mask <= 0, and the partials parts[(r * gridDim.x + b) * 2 + {0, 1}] of
// |R[r]|^2 and |B X[r]|^2.
__global__ void __launch_bounds__(RED_THREADS)
k_lobpcg_residual(int ndof, int vs, const double* __restrict__ GX, const double* __restrict__ KX,
                  const double* __restrict__ mask, const double* __restrict__ theta, double* __restrict__ R,
                  double* __restrict__ parts) {
  __shared__ double red[32 * 2];
  const int r = blockIdx.y;
  const size_t off = (size_t)r * vs;
  const double t = theta[r];
  double s[2] = {0.0, 0.0};
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < ndof; d += gridDim.x * blockDim.x) {
    const double kx = KX[off + d];
    const double e = mask[d] > 0.0 ? GX[off + d] - t * kx : 0.0;
    R[off + d] = e;
    s[0] = fma(e, e, s[0]);
    s[1] = mask[d] > 0.0 ? fma(kx, kx, s[1]) : s[1];
  }
  double o[2];
  block_sum_to_f64<2>(s, red, o);
  if (threadIdx.x == 0) {
    parts[((size_t)r * gridDim.x + blockIdx.x) * 2] = o[0];
    parts[((size_t)r * gridDim.x + blockIdx.x) * 2 + 1] = o[1];
  }
}

// T_lambda of Eq. 3.4 at each element centroid for mode r (phi[r], lam[r]):
// sigma(phi):eps(phi) - lam rho E_e |phi(centroid)|^2, phi(centroid) = the
// mean of the eight nodal vectors (the WHT's constant coefficient / 8).
__global__ void __launch_bounds__(256)
k_eigen_topo(Grid gr, const double* __restrict__ phi, const double* __restrict__ lam, const double* __restrict__ Emod,
             FieldConsts F, double rho, float* __restrict__ out) {
  const int r = blockIdx.y;
  const double* pr = phi + (size_t)r * gr.vs;
  const double lr = lam[r];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < gr.nelem; e += gridDim.x * blockDim.x) {
    const int i = e % gr.nx, j = (e / gr.nx) % gr.ny, k = e / (gr.nx * gr.ny);
    double h[3][8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int n = (i + (a & 1)) + gr.nnx * ((j + ((a >> 1) & 1)) + gr.nny * (k + ((a >> 2) & 1)));
#pragma unroll
      for (int c = 0; c < 3; ++c) h[c][a] = pr[3 * (size_t)n + c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) wht8_fwd(h[c]);
    double eps[6];
    eps[0] = h[0][1] * F.inv4h;
    eps[1] = h[1][2] * F.inv4h;
    eps[2] = h[2][4] * F.inv4h;
    eps[3] = 0.5 * (h[0][2] + h[1][1]) * F.inv4h;
    eps[4] = 0.5 * (h[1][4] + h[2][2]) * F.inv4h;
    eps[5] = 0.5 * (h[2][1] + h[0][4]) * F.inv4h;
    const double E = Emod[e];
    const double tre = eps[0] + eps[1] + eps[2];
    const double la = F.lam * E, mu2 = 2.0 * F.mu * E;
    const double se = (la * tre + mu2 * eps[0]) * eps[0] + (la * tre + mu2 * eps[1]) * eps[1] +
                      (la * tre + mu2 * eps[2]) * eps[2] + 2.0 * mu2 * (eps[3] * eps[3] + eps[4] * eps[4] + eps[5] * eps[5]);
    const double cx = 0.125 * h[0][0], cy = 0.125 * h[1][0], cz = 0.125 * h[2][0];
    out[(size_t)r * gr.nelem + e] = (float)(se - lr * rho * E * (cx * cx + cy * cy + cz * cz));
  }
}

// ---------------------------------------------------------------------------
// Linear buckling (Eq. 3.5): the geometric stiffness K_G of the pre-buckling
// stress, (K + lambda K_G) phi = 0, and the element sensitivity.
// ---------------------------------------------------------------------------

// Stress of the pre-buckling state u0 at each element centroid (xx, yy, zz,
// xy, yz, zx), held constant over the element, times `scale` (the element
// edge h, by which the unit-cube geometric integrals of c_geo scale).
__global__ void __launch_bounds__(256)
k_state_stress(Grid gr, const double* __restrict__ u0, const double* __restrict__ Emod, FieldConsts F, double scale,
               double* __restrict__ S6) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < gr.nelem; e += gridDim.x * blockDim.x) {
    const int i = e % gr.nx, j = (e / gr.nx) % gr.ny, k = e / (gr.nx * gr.ny);
    double eps[6];
    centroid_strain64(gr, u0, i, j, k, F.inv4h, eps);
    const double E = Emod[e];
    const double tre = eps[0] + eps[1] + eps[2];
    const double la = F.lam * E * scale, mu2 = 2.0 * F.mu * E * scale;
#pragma unroll
    for (int q = 0; q < 3; ++q) S6[(size_t)q * gr.nelem + e] = la * tre + mu2 * eps[q];
#pragma unroll
    for (int q = 3; q < 6; ++q) S6[(size_t)q * gr.nelem + e] = mu2 * eps[q];
  }
}

// Element geometric matrix G_e[a][b] = sum_q S_e[q] GEO[q][a][b]: GEO[q] the
// integrals of grad N_a (.) grad N_b over the unit cube for the stress
// components q = xx, yy, zz, xy, yz, zx (off-diagonal pairs summed), set by
// the host; S_e carries the factor h of a cube of edge h.
__constant__ double c_geo[6][8][8];

// Y[r] = sign * K_G X[r], gathered per node over its (up to) eight elements;
// zero on fixed DOFs.  One RHS per blockIdx.y.
__global__ void __launch_bounds__(256)
k_geo_apply(Grid gr, const double* __restrict__ S6, const uint8_t* __restrict__ fixed, double sign,
            const double* __restrict__ X, double* __restrict__ Y) {
  const int r = blockIdx.y;
  const size_t off = (size_t)r * gr.vs;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < gr.nnodes; n += gridDim.x * blockDim.x) {
    const int i = n % gr.nnx, j = (n / gr.nnx) % gr.nny, k = n / (gr.nnx * gr.nny);
    double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int ei = i - 1 + (o & 1), ej = j - 1 + ((o >> 1) & 1), ek = k - 1 + ((o >> 2) & 1);
      if (ei < 0 || ei >= gr.nx || ej < 0 || ej >= gr.ny || ek < 0 || ek >= gr.nz) continue;
      const int e = ei + gr.nx * (ej + gr.ny * ek);
      const int a = 7 - o;   // this node's local index in element e
      double s[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) s[q] = S6[(size_t)q * gr.nelem + e];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        double g = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) g = fma(s[q], c_geo[q][a][b], g);
        const int m = (ei + (b & 1)) + gr.nnx * ((ej + ((b >> 1) & 1)) + gr.nny * (ek + ((b >> 2) & 1)));
        const double* xm = X + off + 3 * (size_t)m;
        acc[0] = fma(g, xm[0], acc[0]);
        acc[1] = fma(g, xm[1], acc[1]);
        acc[2] = fma(g, xm[2], acc[2]);
      }
    }
    const uint8_t fb = fixed ? fixed[n] : 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) Y[off + 3 * (size_t)n + c] = ((fb >> c) & 1) ? 0.0 : sign * acc[c];
  }
}

// Eq. 3.5 per element for mode r (phi[r], lam[r]), with the paper's K_sigma
// read as -K_G: phi_e^T E_e K0 phi_e + lam phi_e^T (G_e kron I3) phi_e.
__global__ void __launch_bounds__(256)
k_buckling_topo(Grid gr, const double* __restrict__ phi, const double* __restrict__ lam,
                const double* __restrict__ Emod, const double* __restrict__ S6, ElemConsts<double> K,
                float* __restrict__ out) {
  const int r = blockIdx.y;
  const double* pr = phi + (size_t)r * gr.vs;
  const double lr = lam[r];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < gr.nelem; e += gridDim.x * blockDim.x) {
    const int i = e % gr.nx, j = (e / gr.nx) % gr.ny, k = e / (gr.nx * gr.ny);
    double v[3][8], w[3][8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int n = (i + (a & 1)) + gr.nnx * ((j + ((a >> 1) & 1)) + gr.nny * (k + ((a >> 2) & 1)));
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c][a] = w[c][a] = pr[3 * (size_t)n + c];
    }
    const double E = Emod[e];
    hex8_apply(w, E, K);   // w = E K0 phi_e
    double s[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) s[q] = S6[(size_t)q * gr.nelem + e];
    double se = 0.0, geo = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
#pragma unroll
      for (int c = 0; c < 3; ++c) se = fma(v[c][a], w[c][a], se);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        double g = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) g = fma(s[q], c_geo[q][a][b], g);
        geo = fma(g, v[0][a] * v[0][b] + v[1][a] * v[1][b] + v[2][a] * v[2][b], geo);
      }
    }
    out[(size_t)r * gr.nelem + e] = (float)(se + lr * geo);
  }
}

}  // namespace afd

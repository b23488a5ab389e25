// Coarse problem of the deflated CG (Sec. 3.5): E = W^T K W for the rigid-body
// modes of agglomerated node groups, built element by element without K
// (only elements whose nodes span several groups, or touch a fixed DOF, carry
// energy for a piecewise rigid field), its FP64 Cholesky factor, and the
// explicit inverse applied once per DPCG iteration.
#pragma once

#include "afd_common.cuh"

namespace afd {

constexpr int COARSE_WARPS = 4;

// Block row G of E: one CTA per group, one warp per element in rounds, a
// private slot per warp, reduced in a fixed order (deterministic).
// E (nc x nc, row-major) must be zeroed before.
__global__ void __launch_bounds__(COARSE_WARPS * 32)
k_coarse_assemble(Grid gr, Groups gp, const double* __restrict__ Emod, const uint8_t* __restrict__ fixed,
                  ElemConsts<double> K, double* __restrict__ Ec) {
  __shared__ double slot[COARSE_WARPS][27 * 36];
  __shared__ double acc[27 * 36];
  const int G = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  const int ilo = gp.g * Gx, ihi = (Gx == gp.ngx - 1) ? gr.nx : gp.g * Gx + gp.g - 1;
  const int jlo = gp.g * Gy, jhi = (Gy == gp.ngy - 1) ? gr.ny : gp.g * Gy + gp.g - 1;
  const int klo = gp.g * Gz, khi = (Gz == gp.ngz - 1) ? gr.nz : gp.g * Gz + gp.g - 1;
  // elements touching the group's nodes
  const int eil = max(ilo - 1, 0), eih = min(ihi, gr.nx - 1);
  const int ejl = max(jlo - 1, 0), ejh = min(jhi, gr.ny - 1);
  const int ekl = max(klo - 1, 0), ekh = min(khi, gr.nz - 1);
  const int lx = eih - eil + 1, ly = ejh - ejl + 1, lz = ekh - ekl + 1;
  const int cnt = lx * ly * lz;
  for (int q = threadIdx.x; q < 27 * 36; q += blockDim.x) acc[q] = 0.0;

  for (int base = 0; base < cnt; base += COARSE_WARPS) {
    for (int q = lane; q < 27 * 36; q += 32) slot[warp][q] = 0.0;
    __syncwarp();
    const int qe = base + warp;
    if (qe < cnt) {
      const int ei = eil + qe % lx, ej = ejl + (qe / lx) % ly, ek = ekl + qe / (lx * ly);
      // groups and fixed bits of the 8 nodes (same in every lane)
      int ng_of[8];
      int fb[8];
      bool active = false;
      bool touches = false;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int i = ei + (a & 1), j = ej + ((a >> 1) & 1), k = ek + ((a >> 2) & 1);
        const int Hx = group_of_axis(i, gp.g, gp.ngx), Hy = group_of_axis(j, gp.g, gp.ngy), Hz = group_of_axis(k, gp.g, gp.ngz);
        ng_of[a] = Hx + gp.ngx * (Hy + gp.ngy * Hz);
        fb[a] = fixed ? fixed[i + gr.nnx * (j + gr.nny * k)] : 0;
        if (ng_of[a] != G || fb[a]) active = true;
        if (ng_of[a] == G) touches = true;
      }
      if (active && touches) {
        const double Ee = Emod[ei + gr.nx * (ej + gr.ny * ek)];
        // tasks: (local node b0 whose group is H, mode col) for each distinct H
        // lane -> task t in [0, 48): H index = t / 6 among distinct groups, col = t % 6
        int distinct[8];
        int nd = 0;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          bool seen = false;
          for (int b = 0; b < nd; ++b) seen |= (distinct[b] == ng_of[a]);
          if (!seen) distinct[nd++] = ng_of[a];
        }
        for (int t = lane; t < nd * 6; t += 32) {
          const int H = distinct[t / 6], col = t % 6;
          const int Hx = H % gp.ngx, Hy = (H / gp.ngx) % gp.ngy, Hz = H / (gp.ngx * gp.ngy);
          const double chx = group_centroid_axis(Hx, gp.g, gp.ngx, gr.nnx, gp.h);
          const double chy = group_centroid_axis(Hy, gp.g, gp.ngy, gr.nny, gp.h);
          const double chz = group_centroid_axis(Hz, gp.g, gp.ngz, gr.nnz, gp.h);
          // column `col` of the masked rigid basis of H on this element
          double v[3][8];
#pragma unroll
          for (int a = 0; a < 8; ++a) {
            const double rx = gp.h * (ei + (a & 1)) - chx;
            const double ry = gp.h * (ej + ((a >> 1) & 1)) - chy;
            const double rz = gp.h * (ek + ((a >> 2) & 1)) - chz;
            double w0 = 0, w1 = 0, w2 = 0;
            if (col < 3) {
              w0 = col == 0; w1 = col == 1; w2 = col == 2;
            } else if (col == 3) {          // e_x x r = (0, -rz, ry)
              w1 = -rz; w2 = ry;
            } else if (col == 4) {          // e_y x r = (rz, 0, -rx)
              w0 = rz; w2 = -rx;
            } else {                         // e_z x r = (-ry, rx, 0)
              w0 = -ry; w1 = rx;
            }
            const bool in = ng_of[a] == H;
            v[0][a] = (in && !(fb[a] & 1)) ? w0 : 0.0;
            v[1][a] = (in && !(fb[a] & 2)) ? w1 : 0.0;
            v[2][a] = (in && !(fb[a] & 4)) ? w2 : 0.0;
          }
          hex8_apply(v, Ee, K);
          // project on G's masked rigid basis (rows of nodes in G, free DOFs)
          const double cgx = group_centroid_axis(Gx, gp.g, gp.ngx, gr.nnx, gp.h);
          const double cgy = group_centroid_axis(Gy, gp.g, gp.ngy, gr.nny, gp.h);
          const double cgz = group_centroid_axis(Gz, gp.g, gp.ngz, gr.nnz, gp.h);
          double o[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
          for (int a = 0; a < 8; ++a) {
            if (ng_of[a] != G) continue;
            const double fx = (fb[a] & 1) ? 0.0 : v[0][a];
            const double fy = (fb[a] & 2) ? 0.0 : v[1][a];
            const double fz = (fb[a] & 4) ? 0.0 : v[2][a];
            const double rx = gp.h * (ei + (a & 1)) - cgx;
            const double ry = gp.h * (ej + ((a >> 1) & 1)) - cgy;
            const double rz = gp.h * (ek + ((a >> 2) & 1)) - cgz;
            o[0] += fx;
            o[1] += fy;
            o[2] += fz;
            o[3] += ry * fz - rz * fy;
            o[4] += rz * fx - rx * fz;
            o[5] += rx * fy - ry * fx;
          }
          const int sidx = (Hx - Gx + 1) + 3 * (Hy - Gy + 1) + 9 * (Hz - Gz + 1);
#pragma unroll
          for (int r = 0; r < 6; ++r) slot[warp][sidx * 36 + r * 6 + col] = o[r];
        }
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 27 * 36; q += blockDim.x) {
      double s = acc[q];
      for (int w = 0; w < COARSE_WARPS; ++w) s += slot[w][q];
      acc[q] = s;
    }
    __syncthreads();
  }
  const int nc = 6 * gp.ng;
  for (int q = threadIdx.x; q < 27 * 36; q += blockDim.x) {
    const int sidx = q / 36, r = (q % 36) / 6, col = q % 6;
    const int Hx = Gx + sidx % 3 - 1, Hy = Gy + (sidx / 3) % 3 - 1, Hz = Gz + sidx / 9 - 1;
    if (Hx < 0 || Hy < 0 || Hz < 0 || Hx >= gp.ngx || Hy >= gp.ngy || Hz >= gp.ngz) continue;
    const int H = Hx + gp.ngx * (Hy + gp.ngy * Hz);
    Ec[(size_t)(6 * G + r) * nc + 6 * H + col] = acc[q];
  }
}

// ---------------------------------------------------------------------------
// Dense FP64 Cholesky, right-looking, block NB (lower triangle, row-major).
// ---------------------------------------------------------------------------
constexpr int CH_NB = 32;

// Largest diagonal entry of A (single block), for the relative pivot test.
__global__ void k_max_diag(const double* A, int n, double* out) {
  __shared__ double sh[256];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(A[(size_t)i * n + i]));
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// Factor the diagonal block at k0 (size nb <= CH_NB) in shared memory.  A
// pivot <= 1e-12 * max diag (or NaN) marks the coarse matrix singular (no
// supports leave the rigid modes of the whole body in the coarse space).
__global__ void k_potrf_diag(double* A, int n, int k0, const double* dmax, int* status) {
  __shared__ double s[CH_NB][CH_NB + 1];
  const int nb = min(CH_NB, n - k0);
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) s[q / nb][q % nb] = A[(size_t)(k0 + q / nb) * n + k0 + q % nb];
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      const double d = s[j][j];
      if (!(d > 1e-12 * (*dmax)) || !isfinite(d)) {
        *status = -4;
        s[j][j] = 1.0;
      } else {
        s[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    const double djj = s[j][j];
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) s[i][j] /= djj;
    __syncthreads();
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
      const int i = q / nb, c = q % nb;
      if (i > j && c > j && c <= i) s[i][c] -= s[i][j] * s[c][j];
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
    const int i = q / nb, c = q % nb;
    A[(size_t)(k0 + i) * n + k0 + c] = (c <= i) ? s[i][c] : 0.0;
  }
}

// L_ik = A_ik L_kk^{-T} for every row i >= k0 + nb: one thread per row.
__global__ void k_trsm_panel(double* A, int n, int k0) {
  __shared__ double L[CH_NB][CH_NB + 1];
  const int nb = min(CH_NB, n - k0);
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) L[q / nb][q % nb] = A[(size_t)(k0 + q / nb) * n + k0 + q % nb];
  __syncthreads();
  const int i = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[CH_NB];
  double* row = A + (size_t)i * n + k0;
  for (int j = 0; j < nb; ++j) {
    double v = row[j];
    for (int m = 0; m < j; ++m) v -= x[m] * L[j][m];
    x[j] = v / L[j][j];
  }
  for (int j = 0; j < nb; ++j) row[j] = x[j];
}

// A_ij -= sum_m L_im L_jm over the panel columns [k0, k0+nb) for the trailing
// lower triangle; 32x32 output tile per CTA (256 threads, 4 outputs each).
__global__ void k_syrk_update(double* A, int n, int k0) {
  __shared__ double Li[32][CH_NB + 1];
  __shared__ double Lj[32][CH_NB + 1];
  const int nb = min(CH_NB, n - k0);
  const int t0 = k0 + nb;
  const int nt = (n - t0 + 31) / 32;
  // blockIdx.x enumerates lower tiles (ti >= tj)
  int b = blockIdx.x, ti = 0;
  while (b >= ti + 1) { b -= ti + 1; ++ti; }
  const int tj = b;
  if (ti >= nt) return;
  const int i0 = t0 + 32 * ti, j0 = t0 + 32 * tj;
  for (int q = threadIdx.x; q < 32 * nb; q += blockDim.x) {
    const int r = q / nb, c = q % nb;
    Li[r][c] = (i0 + r < n) ? A[(size_t)(i0 + r) * n + k0 + c] : 0.0;
    Lj[r][c] = (j0 + r < n) ? A[(size_t)(j0 + r) * n + k0 + c] : 0.0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q / 32, c = q % 32;
    const int i = i0 + r, j = j0 + c;
    if (i >= n || j >= n || j > i) continue;
    double s = 0.0;
    for (int m = 0; m < nb; ++m) s = fma(Li[r][m], Lj[c][m], s);
    A[(size_t)i * n + j] -= s;
  }
}

// U = L^T (row-major) so that column k of L is a contiguous row of U.
__global__ void k_transpose(const double* L, double* U, int n) {
  __shared__ double t[32][33];
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 32 + threadIdx.y;
  for (int r = 0; r < 32; r += 8)
    if (x < n && y + r < n) t[threadIdx.y + r][threadIdx.x] = L[(size_t)(y + r) * n + x];
  __syncthreads();
  const int xo = blockIdx.y * 32 + threadIdx.x, yo = blockIdx.x * 32 + threadIdx.y;
  for (int r = 0; r < 32; r += 8)
    if (xo < n && yo + r < n) U[(size_t)(yo + r) * n + xo] = t[threadIdx.x][threadIdx.y + r];
}

// Column j of L^{-1} (lower): solve L x = e_j by column-oriented forward
// substitution, reading column k of L as row k of U = L^T; one CTA per
// column, x in shared memory (n doubles).
__global__ void k_trtri_cols(const double* U, double* Linv, int n) {
  extern __shared__ double x[];
  const int j = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = (i == j) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = j; k < n; ++k) {
    const double* uk = U + (size_t)k * n;
    const double xk = x[k] / uk[k];
    __syncthreads();
    if (threadIdx.x == 0) x[k] = xk;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) x[i] -= uk[i] * xk;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) Linv[(size_t)i * n + j] = (i >= j) ? x[i] : 0.0;
}

// Einv = Linv^T Linv: Einv_ij = sum_{k >= max(i,j)} Linv_ki Linv_kj; 32x32 tiles.
__global__ void k_gram(const double* Linv, double* Einv, int n) {
  __shared__ double A[32][33];
  __shared__ double B[32][33];
  const int i0 = 32 * blockIdx.y, j0 = 32 * blockIdx.x;
  const int r = threadIdx.x / 32, c = threadIdx.x % 32;  // 1024 threads
  double s = 0.0;
  const int kstart = (max(i0, j0) / 32) * 32;
  for (int k0 = kstart; k0 < n; k0 += 32) {
    A[r][c] = (k0 + r < n && i0 + c < n) ? Linv[(size_t)(k0 + r) * n + i0 + c] : 0.0;
    B[r][c] = (k0 + r < n && j0 + c < n) ? Linv[(size_t)(k0 + r) * n + j0 + c] : 0.0;
    __syncthreads();
#pragma unroll 8
    for (int m = 0; m < 32; ++m) s = fma(A[m][r], B[m][c], s);
    __syncthreads();
  }
  if (i0 + r < n && j0 + c < n) Einv[(size_t)(i0 + r) * n + j0 + c] = s;
}

}  // namespace afd

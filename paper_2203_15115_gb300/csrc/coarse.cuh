// Coarse problem of the deflated CG (Sec. 3.5): E = W^T K W for the rigid-body
// modes of agglomerated node groups, built element by element without K
// (only elements whose nodes span several groups, or touch a fixed DOF, carry
// energy for a piecewise rigid field), its FP64 Cholesky factor, and the
// explicit inverse applied once per DPCG iteration.
#pragma once

#include "afd_common.cuh"

namespace afd {

// One 6x6 block E_GH = W_G^T K W_H per CTA (blockIdx.x = G, blockIdx.y = the
// neighbour slot of H).  Only elements with nodes in both groups contribute,
// and for G == H only those whose nodes leave the group or touch a fixed DOF
// (W_G is a rigid motion on the others, which K annihilates).  Element math in
// TC (float for the mixed path, double for the FP64 path), per-thread sums in
// TC, block reduction in FP64 in a fixed order.  Every block of Ec is written.
constexpr int COARSE_THREADS = 256;

template <typename TC>
__global__ void __launch_bounds__(COARSE_THREADS)
k_coarse_block(Grid gr, Groups gp, const double* __restrict__ Emod, const uint8_t* __restrict__ fixed,
               ElemConsts<TC> K, double* __restrict__ Ec) {
  __shared__ double red[32 * 36];
  const int G = blockIdx.x, slot = blockIdx.y;
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  const int Hx = Gx + slot % 3 - 1, Hy = Gy + (slot / 3) % 3 - 1, Hz = Gz + slot / 9 - 1;
  if (Hx < 0 || Hy < 0 || Hz < 0 || Hx >= gp.ngx || Hy >= gp.ngy || Hz >= gp.ngz) return;
  const int H = Hx + gp.ngx * (Hy + gp.ngy * Hz);
  auto lohi = [&](int X, int ng, int n, int& lo, int& hi) {
    lo = gp.g * X;
    hi = (X == ng - 1) ? n : gp.g * X + gp.g - 1;
  };
  int gxl, gxh, gyl, gyh, gzl, gzh, hxl, hxh, hyl, hyh, hzl, hzh;
  lohi(Gx, gp.ngx, gr.nx, gxl, gxh); lohi(Gy, gp.ngy, gr.ny, gyl, gyh); lohi(Gz, gp.ngz, gr.nz, gzl, gzh);
  lohi(Hx, gp.ngx, gr.nx, hxl, hxh); lohi(Hy, gp.ngy, gr.ny, hyl, hyh); lohi(Hz, gp.ngz, gr.nz, hzl, hzh);
  // elements with a node in both boxes
  const int eil = max(max(gxl, hxl) - 1, 0), eih = min(min(gxh, hxh), gr.nx - 1);
  const int ejl = max(max(gyl, hyl) - 1, 0), ejh = min(min(gyh, hyh), gr.ny - 1);
  const int ekl = max(max(gzl, hzl) - 1, 0), ekh = min(min(gzh, hzh), gr.nz - 1);
  const int lx = eih - eil + 1, ly = ejh - ejl + 1, lz = ekh - ekl + 1;
  const int cnt = (lx > 0 && ly > 0 && lz > 0) ? lx * ly * lz : 0;
  const TC cgx = (TC)(0.5 * gp.h * (gxl + gxh)), cgy = (TC)(0.5 * gp.h * (gyl + gyh)), cgz = (TC)(0.5 * gp.h * (gzl + gzh));
  const TC chx = (TC)(0.5 * gp.h * (hxl + hxh)), chy = (TC)(0.5 * gp.h * (hyl + hyh)), chz = (TC)(0.5 * gp.h * (hzl + hzh));
  const TC hh = (TC)gp.h;
  TC acc[36];
#pragma unroll
  for (int q = 0; q < 36; ++q) acc[q] = TC(0);
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int ei = eil + q % lx, ej = ejl + (q / lx) % ly, ek = ekl + q / (lx * ly);
    bool inG[8], inH[8];
    int fb[8];
    bool anyG = false, anyH = false, leaves = false, anyfix = false;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int i = ei + (a & 1), j = ej + ((a >> 1) & 1), k = ek + ((a >> 2) & 1);
      inG[a] = i >= gxl && i <= gxh && j >= gyl && j <= gyh && k >= gzl && k <= gzh;
      inH[a] = i >= hxl && i <= hxh && j >= hyl && j <= hyh && k >= hzl && k <= hzh;
      fb[a] = fixed ? fixed[i + gr.nnx * (j + gr.nny * k)] : 0;
      anyG |= inG[a];
      anyH |= inH[a];
      leaves |= !inG[a];
      anyfix |= (inG[a] && fb[a]) || (inH[a] && fb[a]);
    }
    if (!anyG || !anyH) continue;
    if (G == H && !leaves && !anyfix) continue;
    const TC Ee = (TC)Emod[ei + gr.nx * (ej + gr.ny * ek)];
#pragma unroll 1
    for (int col = 0; col < 6; ++col) {
      TC v[3][8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const TC rx = hh * (TC)(ei + (a & 1)) - chx;
        const TC ry = hh * (TC)(ej + ((a >> 1) & 1)) - chy;
        const TC rz = hh * (TC)(ek + ((a >> 2) & 1)) - chz;
        TC w0 = 0, w1 = 0, w2 = 0;
        if (col == 0) w0 = 1;
        else if (col == 1) w1 = 1;
        else if (col == 2) w2 = 1;
        else if (col == 3) { w1 = -rz; w2 = ry; }    // e_x x r
        else if (col == 4) { w0 = rz; w2 = -rx; }    // e_y x r
        else { w0 = -ry; w1 = rx; }                  // e_z x r
        v[0][a] = (inH[a] && !(fb[a] & 1)) ? w0 : TC(0);
        v[1][a] = (inH[a] && !(fb[a] & 2)) ? w1 : TC(0);
        v[2][a] = (inH[a] && !(fb[a] & 4)) ? w2 : TC(0);
      }
      hex8_apply(v, Ee, K);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        if (!inG[a]) continue;
        const TC fx = (fb[a] & 1) ? TC(0) : v[0][a];
        const TC fy = (fb[a] & 2) ? TC(0) : v[1][a];
        const TC fz = (fb[a] & 4) ? TC(0) : v[2][a];
        const TC rx = hh * (TC)(ei + (a & 1)) - cgx;
        const TC ry = hh * (TC)(ej + ((a >> 1) & 1)) - cgy;
        const TC rz = hh * (TC)(ek + ((a >> 2) & 1)) - cgz;
        TC* o = acc;  // o[r * 6 + col]
        switch (col) {
#define AFD_ACC(C)                                   \
  case C:                                            \
    o[0 * 6 + C] += fx;                              \
    o[1 * 6 + C] += fy;                              \
    o[2 * 6 + C] += fz;                              \
    o[3 * 6 + C] += ry * fz - rz * fy;               \
    o[4 * 6 + C] += rz * fx - rx * fz;               \
    o[5 * 6 + C] += rx * fy - ry * fx;               \
    break;
          AFD_ACC(0) AFD_ACC(1) AFD_ACC(2) AFD_ACC(3) AFD_ACC(4) AFD_ACC(5)
#undef AFD_ACC
        }
      }
    }
  }
  double o[36];
  block_sum_to_f64<36>(acc, red, o);
  if (threadIdx.x == 0) {
    const int nc = 6 * gp.ng;
#pragma unroll
    for (int q = 0; q < 36; ++q) Ec[(size_t)(6 * G + q / 6) * nc + 6 * H + q % 6] = o[q];
  }
}

// The same blocks from the cut-element records of each group G (the shells
// of the coarse right-hand side: k_build_cut_recs).  Every element that
// couples G with a neighbour H, or on which W_G is not a rigid motion, is one
// of G's records.  Blocks:
//   blockIdx.y < nself: a share of E_GG, its 36 sums left in part[G][share];
//     the group's last share adds the shares in order (deterministic);
//   blockIdx.y = nself + s: E_GH for the neighbour slot 14 + s (the 13
//     neighbours after G in group order), written with its transpose E_HG.
// Element math in TC, per-thread sums in TC, block sums in FP64, as in
// k_coarse_block.
template <typename TC>
__global__ void __launch_bounds__(COARSE_THREADS)
k_coarse_cut(Grid gr, Groups gp, int nself, const uint4* __restrict__ cut, const long long* __restrict__ cut_off,
             const double* __restrict__ Emod, ElemConsts<TC> K, double* __restrict__ Ec, double* __restrict__ part,
             unsigned int* __restrict__ counter) {
  __shared__ double red[32 * 36];
  __shared__ bool s_last;
  const int G = blockIdx.x, y = blockIdx.y;
  const bool self = y < nself;
  const int slot = self ? 13 : 14 + (y - nself);
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  const int Hx = Gx + slot % 3 - 1, Hy = Gy + (slot / 3) % 3 - 1, Hz = Gz + slot / 9 - 1;
  if (Hx < 0 || Hy < 0 || Hz < 0 || Hx >= gp.ngx || Hy >= gp.ngy || Hz >= gp.ngz) return;
  const int H = Hx + gp.ngx * (Hy + gp.ngy * Hz);
  auto lohi = [&](int X, int ng, int n, int& lo, int& hi) {
    lo = gp.g * X;
    hi = (X == ng - 1) ? n : gp.g * X + gp.g - 1;
  };
  int gxl, gxh, gyl, gyh, gzl, gzh, hxl, hxh, hyl, hyh, hzl, hzh;
  lohi(Gx, gp.ngx, gr.nx, gxl, gxh); lohi(Gy, gp.ngy, gr.ny, gyl, gyh); lohi(Gz, gp.ngz, gr.nz, gzl, gzh);
  lohi(Hx, gp.ngx, gr.nx, hxl, hxh); lohi(Hy, gp.ngy, gr.ny, hyl, hyh); lohi(Hz, gp.ngz, gr.nz, hzl, hzh);
  const TC cgx = (TC)(0.5 * gp.h * (gxl + gxh)), cgy = (TC)(0.5 * gp.h * (gyl + gyh)), cgz = (TC)(0.5 * gp.h * (gzl + gzh));
  const TC chx = (TC)(0.5 * gp.h * (hxl + hxh)), chy = (TC)(0.5 * gp.h * (hyl + hyh)), chz = (TC)(0.5 * gp.h * (hzl + hzh));
  const TC hh = (TC)gp.h;
  const long long base = cut_off[G];
  const int cnt = (int)(cut_off[G + 1] - base);
  int tb = 0, te = cnt;
  if (self) {
    const int per = (cnt + nself - 1) / nself;
    tb = y * per;
    te = min(tb + per, cnt);
  }
  TC acc[36];
#pragma unroll
  for (int q = 0; q < 36; ++q) acc[q] = TC(0);
  for (int t = tb + threadIdx.x; t < te; t += blockDim.x) {
    const uint4 rec = cut[base + t];
    const int ei = gxl - 1 + (int)(rec.z & 1023u), ej = gyl - 1 + (int)((rec.z >> 10) & 1023u),
              ek = gzl - 1 + (int)((rec.z >> 20) & 1023u);
    const unsigned ing = rec.w >> 24, fbits = rec.w & 0xFFFFFFu;
    unsigned inh = ing;
    if (!self) {
      inh = 0;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int i = ei + (a & 1), j = ej + ((a >> 1) & 1), k = ek + ((a >> 2) & 1);
        if (i >= hxl && i <= hxh && j >= hyl && j <= hyh && k >= hzl && k <= hzh) inh |= 1u << a;
      }
      if (!inh) continue;
    }
    const TC Ee = (TC)Emod[rec.y];
#pragma unroll 1
    for (int col = 0; col < 6; ++col) {
      TC v[3][8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const TC rx = hh * (TC)(ei + (a & 1)) - chx;
        const TC ry = hh * (TC)(ej + ((a >> 1) & 1)) - chy;
        const TC rz = hh * (TC)(ek + ((a >> 2) & 1)) - chz;
        TC w0 = 0, w1 = 0, w2 = 0;
        if (col == 0) w0 = 1;
        else if (col == 1) w1 = 1;
        else if (col == 2) w2 = 1;
        else if (col == 3) { w1 = -rz; w2 = ry; }    // e_x x r
        else if (col == 4) { w0 = rz; w2 = -rx; }    // e_y x r
        else { w0 = -ry; w1 = rx; }                  // e_z x r
        const unsigned fb = (fbits >> (3 * a)) & 7u;
        const bool h_a = (inh >> a) & 1u;
        v[0][a] = (h_a && !(fb & 1)) ? w0 : TC(0);
        v[1][a] = (h_a && !(fb & 2)) ? w1 : TC(0);
        v[2][a] = (h_a && !(fb & 4)) ? w2 : TC(0);
      }
      hex8_apply(v, Ee, K);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        if (!((ing >> a) & 1u)) continue;
        const unsigned fb = (fbits >> (3 * a)) & 7u;
        const TC fx = (fb & 1) ? TC(0) : v[0][a];
        const TC fy = (fb & 2) ? TC(0) : v[1][a];
        const TC fz = (fb & 4) ? TC(0) : v[2][a];
        const TC rx = hh * (TC)(ei + (a & 1)) - cgx;
        const TC ry = hh * (TC)(ej + ((a >> 1) & 1)) - cgy;
        const TC rz = hh * (TC)(ek + ((a >> 2) & 1)) - cgz;
        TC* o = acc;  // o[r * 6 + col]
        switch (col) {
#define AFD_ACC(C)                                   \
  case C:                                            \
    o[0 * 6 + C] += fx;                              \
    o[1 * 6 + C] += fy;                              \
    o[2 * 6 + C] += fz;                              \
    o[3 * 6 + C] += ry * fz - rz * fy;               \
    o[4 * 6 + C] += rz * fx - rx * fz;               \
    o[5 * 6 + C] += rx * fy - ry * fx;               \
    break;
          AFD_ACC(0) AFD_ACC(1) AFD_ACC(2) AFD_ACC(3) AFD_ACC(4) AFD_ACC(5)
#undef AFD_ACC
        }
      }
    }
  }
  double o[36];
  block_sum_to_f64<36>(acc, red, o);
  const int nc = 6 * gp.ng;
  if (!self) {
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < 36; ++q) {
        Ec[(size_t)(6 * G + q / 6) * nc + 6 * H + q % 6] = o[q];
        Ec[(size_t)(6 * H + q % 6) * nc + 6 * G + q / 6] = o[q];
      }
    }
    return;
  }
  double* mine = part + ((size_t)G * nself + y) * 36;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 36; ++q) mine[q] = o[q];
    __threadfence();
    s_last = atomicAdd(&counter[G], 1u) == (unsigned)nself - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 36) {
    const double* pp = part + (size_t)G * nself * 36;
    double v = 0.0;
    for (int s2 = 0; s2 < nself; ++s2) v += pp[s2 * 36 + threadIdx.x];
    Ec[(size_t)(6 * G + threadIdx.x / 6) * nc + 6 * G + threadIdx.x % 6] = v;
  }
  if (threadIdx.x == 0) counter[G] = 0u;
}

// ---------------------------------------------------------------------------
// Dense inverse of the SPD coarse matrix by blocked Gauss-Jordan sweeps:
// sweeping block K replaces A_KK by -A_KK^{-1}, A_iK by A_iK A_KK^{-1},
// A_Kj by A_KK^{-1} A_Kj and A_ij by A_ij - A_iK A_KK^{-1} A_Kj; after every
// block has been swept the matrix holds -A^{-1}.  No pivoting (SPD: every
// swept diagonal block is a Schur complement, hence SPD).  n^3 multiply-adds,
// n / GJ_NB sequential steps of three launches, each fully parallel.
// ---------------------------------------------------------------------------
constexpr int GJ_NB = 32;

template <typename T>
__global__ void k_convert_dense(size_t n, const double* __restrict__ a, T* __restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = (T)a[i];
}

// dinv[i] = 1 / sqrt(a_ii) of a dense FP64 matrix (NaN for a diagonal <= 0).
__global__ void k_diag_rsqrt(int n, const double* __restrict__ a, double* __restrict__ dinv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double d = a[(size_t)i * n + i];
    dinv[i] = d > 0.0 ? 1.0 / sqrt(d) : (double)NAN;
  }
}

// b = D^{-1/2} a D^{-1/2} (D = diag a, dinv = its inverse square roots) in
// type T: the coarse matrix with unit diagonal, so that the inverse does not
// lose the small rigid modes of groups whose elements are mostly void.  A
// diagonal <= 0 gives NaN, which the pivot test reports as singular.
// (n <= 8192, so n * n and the indices fit in 32 bits.)
template <typename T>
__global__ void k_scale_dense(int n, const double* __restrict__ a, const double* __restrict__ dinv,
                              T* __restrict__ b) {
  const unsigned nn = (unsigned)n * (unsigned)n;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < nn; q += gridDim.x * blockDim.x) {
    const unsigned i = q / (unsigned)n, j = q - i * (unsigned)n;
    b[q] = (T)(a[q] * dinv[i] * dinv[j]);
  }
}

// b <- D^{-1/2} b D^{-1/2}: the inverse of the scaled matrix back to the
// inverse of a.
template <typename T>
__global__ void k_unscale_dense(int n, const double* __restrict__ dinv, T* __restrict__ b) {
  const unsigned nn = (unsigned)n * (unsigned)n;
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < nn; q += gridDim.x * blockDim.x) {
    const unsigned i = q / (unsigned)n, j = q - i * (unsigned)n;
    b[q] = (T)((double)b[q] * dinv[i] * dinv[j]);
  }
}

// Invert the nb x nb diagonal block at k0 by unblocked sweeps held in the
// registers of one warp: lane i keeps row i of the block, the pivot column is
// in every lane's own registers and the pivot row arrives by shuffles, so a
// sweep costs no barrier.  P = A_KK^{-1} (nb x nb).  Rows and columns beyond
// nb are an identity (pivot 1, no coupling).  A pivot <= rel * (*dmax) (or
// NaN) sets *status (the sweep continues with pivot 1).  The block is read
// row by row (coalesced) through shared memory, and the pivot test runs in
// the working type, off the FP64 unit.
template <typename T> struct FiniteMax;
template <> struct FiniteMax<float> { static constexpr float v = 3.40282347e38f; };
template <> struct FiniteMax<double> { static constexpr double v = 1.7976931348623157e308; };

template <typename T>
__global__ void __launch_bounds__(32) k_gj_pivot(const T* A, int n, int k0, T* P, const double* dmax, double rel,
                                                 int* status) {
  __shared__ T blk[GJ_NB][GJ_NB + 1];
  const int nb = min(GJ_NB, n - k0);
  const int i = threadIdx.x;
#pragma unroll 8
  for (int r = 0; r < GJ_NB; ++r)
    blk[r][i] = (r < nb && i < nb) ? A[(size_t)(k0 + r) * n + k0 + i] : (r == i ? T(1) : T(0));
  __syncwarp();
  T s[GJ_NB];
#pragma unroll
  for (int j = 0; j < GJ_NB; ++j) s[j] = blk[i][j];
  const T thr = (T)(rel * (*dmax));
  bool bad = false;
#pragma unroll
  for (int p = 0; p < GJ_NB; ++p) {
    const T colp = s[p];   // this row's entry in the pivot column
    T d = __shfl_sync(0xffffffffu, colp, p);
    if (p < nb && !(d > thr && d <= FiniteMax<T>::v)) {   // too small, NaN or infinite
      bad = true;
      d = T(1);
    }
    const T inv = T(1) / d;
#pragma unroll
    for (int j = 0; j < GJ_NB; ++j) {
      const T rowp = __shfl_sync(0xffffffffu, s[j], p);
      T v;
      if (i == p) v = (j == p) ? -inv : rowp * inv;
      else v = (j == p) ? colp * inv : s[j] - colp * rowp * inv;
      s[j] = v;
    }
  }
  // s = -A_KK^{-1}
  if (i < nb) {
#pragma unroll
    for (int j = 0; j < GJ_NB; ++j)
      if (j < nb) P[i * nb + j] = -s[j];
  }
  if (bad && i == 0) *status = -4;
}

// B[i][m] = sum_t A[i][k0+t] P[t][m] for every row i outside K (rows of K
// untouched), and R[t][j] = A[k0+t][j] (a copy of the block row).
template <typename T>
__global__ void __launch_bounds__(256) k_gj_panel(const T* __restrict__ A, int n, int k0, const T* __restrict__ P,
                                                  T* __restrict__ B, T* __restrict__ R) {
  __shared__ T Ps[GJ_NB][GJ_NB];
  const int nb = min(GJ_NB, n - k0);
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) Ps[q / nb][q % nb] = P[q];
  __syncthreads();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  // rows: one thread per (row, m)
  if (idx < n * nb) {
    const int i = idx / nb, m = idx % nb;
    if (i < k0 || i >= k0 + nb) {
      T s = T(0);
      const T* ai = A + (size_t)i * n + k0;
      for (int t = 0; t < nb; ++t) s = fma(ai[t], Ps[t][m], s);
      B[(size_t)i * GJ_NB + m] = s;
    }
    R[(size_t)m * n + i] = A[(size_t)(k0 + m) * n + i];
  }
}

// Schur update and the swept block row/column; 32x32 tile per CTA.
// When `last`, the result is negated so that A holds the inverse.
template <typename T>
__global__ void __launch_bounds__(256) k_gj_update(T* __restrict__ A, int n, int k0, const T* __restrict__ P,
                                                   const T* __restrict__ B, const T* __restrict__ R, int last) {
  __shared__ T Bs[32][GJ_NB + 1];
  __shared__ T Rs[GJ_NB][32 + 1];
  const int nb = min(GJ_NB, n - k0);
  const int i0 = 32 * blockIdx.y, j0 = 32 * blockIdx.x;
  for (int q = threadIdx.x; q < 32 * GJ_NB; q += blockDim.x) {
    const int r = q / GJ_NB, m = q % GJ_NB;
    const int i = i0 + r;
    Bs[r][m] = (i < n && m < nb && (i < k0 || i >= k0 + nb)) ? B[(size_t)i * GJ_NB + m] : T(0);
    const int jm = q / 32, jc = q % 32;
    Rs[jm][jc] = (jm < nb && j0 + jc < n) ? R[(size_t)jm * n + j0 + jc] : T(0);
  }
  __syncthreads();
  const T sg = last ? T(-1) : T(1);
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q / 32, c = q % 32;
    const int i = i0 + r, j = j0 + c;
    if (i >= n || j >= n) continue;
    const bool iK = i >= k0 && i < k0 + nb, jK = j >= k0 && j < k0 + nb;
    T v;
    if (iK && jK) {
      v = -P[(i - k0) * nb + (j - k0)];
    } else if (jK) {
      v = Bs[r][j - k0];
    } else if (iK) {
      v = B[(size_t)j * GJ_NB + (i - k0)];  // (A_KK^{-1} A_Kj)_i = (A_jK A_KK^{-1})_i by symmetry
    } else {
      T s = A[(size_t)i * n + j];
#pragma unroll 8
      for (int m = 0; m < GJ_NB; ++m) s = fma(-Bs[r][m], Rs[m][c], s);
      v = s;
    }
    A[(size_t)i * n + j] = sg * v;
  }
}

// Largest |diagonal| of a dense double matrix (single block).
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

}  // namespace afd

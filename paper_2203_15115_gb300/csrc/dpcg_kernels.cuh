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
constexpr int CSTEP_THREADS = 256;  // threads of a coarse-step block: one warp per row of the inverse (measured against 64 and 128)

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
  // rho of the previous iteration and the iteration count, in two slots by
  // the iteration's parity (dpcg_iteration_start reads slot par, writes par^1)
  double rzs[2];
  int its[2];
};

// Where the stencil that starts an iteration finds the partial sums of the
// previous one: (r.z, r.r) per vector-update block and (W^T r).mu per
// coarse-step block, and the parity of the iteration.
struct IterPartials {
  const double* upd;   // [rhs][nupd][2]
  int nupd;
  const double* cd;    // [rhs][ncd]
  int ncd;
  int par;
};

// Block-wide sum in a fixed order (per-thread strided sums, warp tree, then
// warps in order); any blockDim.x that is a multiple of 32, up to 1024.  The
// result is returned to every thread.
__device__ inline double block_sum_bcast(double s) {
  __shared__ double sh[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s = warp_sum(s);
  if (lane == 0) sh[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    sh[32] = t;
  }
  __syncthreads();
  const double out = sh[32];
  __syncthreads();
  return out;
}

// Start of iteration i of the DPCG loop, taken by every CTA of the stencil
// that applies K to the next search direction: rho_i = r.z + (W^T r).mu and
// r.r from the partials of the vector update and the coarse step of
// iteration i-1, the stopping test (converged, not finite, or out of
// iterations) and beta_i = rho_i / rho_{i-1}.  Every CTA sums the same
// partials in the same order and takes the same decision; CTA (0, 0) records
// it in the state.  rho_{i-1} and i are read from slot par and rho_i, i+1
// written to slot par^1, so the recording never meets another CTA's read.
// Returns false (in every thread) when the RHS stops.
__device__ inline bool dpcg_iteration_start(CGState* st, int rhs, int* done_flags, const IterPartials& ip,
                                            double& beta) {
  __shared__ double red[32 * 3];
  __shared__ int s_go;
  __shared__ double s_beta;
  // the state's fields are loaded with the partials, not after their sum
  double rho_old = 0.0, target2 = 0.0;
  int it = 0, max_iters = 0;
  if (threadIdx.x == 0) {
    const CGState& S = st[rhs];
    rho_old = S.rzs[ip.par];
    it = S.its[ip.par];
    target2 = S.target2;
    max_iters = S.max_iters;
  }
  double ps[3] = {0.0, 0.0, 0.0};
  const double2* up = (const double2*)(ip.upd + (size_t)rhs * ip.nupd * 2);
  for (int i = threadIdx.x; i < ip.nupd; i += blockDim.x) {
    const double2 v = up[i];
    ps[0] += v.x;
    ps[1] += v.y;
  }
  const double* cd = ip.cd + (size_t)rhs * ip.ncd;
  for (int i = threadIdx.x; i < ip.ncd; i += blockDim.x) ps[2] += cd[i];
  double o[3];
  block_sum_to_f64<3>(ps, red, o);
  if (threadIdx.x == 0) {
    CGState& S = st[rhs];
    const double rho = o[0] + o[2], rr = o[1];
    int status = 1;
    if (!isfinite(rr) || !isfinite(rho)) status = -5;
    else if (rr <= target2) status = 0;
    else if (it >= max_iters) status = -3;
    const bool lead = blockIdx.x == 0 && blockIdx.y == 0;
    const double b = rho / rho_old;
    if (lead) {
      S.rz = rho;
      S.rr = rr;
      S.iters = it;
      if (status != 1) {
        S.status = status;
        S.done = 1;
        if (done_flags) done_flags[rhs] = 1;
      } else {
        S.beta = b;
        S.rzs[ip.par ^ 1] = rho;
        S.its[ip.par ^ 1] = it + 1;
      }
    }
    s_go = status == 1;
    s_beta = b;
  }
  __syncthreads();
  beta = s_beta;
  return s_go != 0;
}

// Sum nparts partials (stride `stride`, component `comp`) of one RHS in a fixed order.
__device__ inline double sum_partials(const double* p, int nparts, int stride, int comp) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += p[(size_t)i * stride + comp];
  return block_sum_bcast(s);
}

// ---------------------------------------------------------------------------
// Deflation (Sec. 3.5; coarse space = rigid-body modes of agglomerated groups)
// ---------------------------------------------------------------------------

// Node-plane range [lo, hi] of group X along an axis with n elements.
__device__ __forceinline__ void group_range(int X, int g, int ng, int n, int& lo, int& hi) {
  lo = g * X;
  hi = (X == ng - 1) ? n : g * X + g - 1;
}

// W^T of one or two vectors: for each group G the sums over its free DOFs of
// (v, r x v), r = x_node - c_G (force and moment about the group centroid).
// out_a[rhs][6G+q] = (W^T a)_G, out_b = W^T b when b is given.  One block per
// (group, rhs); FP64 output.  (Used by the deflated start and the tests.)
template <typename T>
__global__ void __launch_bounds__(256)
k_restrict(Grid gr, Groups gp, const T* __restrict__ a, const T* __restrict__ b, const uint8_t* __restrict__ fixed,
           double* __restrict__ out_a, double* __restrict__ out_b, const CGState* st) {
  __shared__ double red[32 * 12];
  const int G = blockIdx.x, rhs = blockIdx.y;
  if (st && st[rhs].done) return;
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  int ilo, ihi, jlo, jhi, klo, khi;
  group_range(Gx, gp.g, gp.ngx, gr.nx, ilo, ihi);
  group_range(Gy, gp.g, gp.ngy, gr.ny, jlo, jhi);
  group_range(Gz, gp.g, gp.ngz, gr.nz, klo, khi);
  const T hh = (T)(0.5 * gp.h);
  const int lx = ihi - ilo + 1, ly = jhi - jlo + 1, lz = khi - klo + 1;
  const int cnt = lx * ly * lz;
  const size_t off = (size_t)rhs * gr.vs;
  T s[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) s[q] = T(0);
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int i = ilo + q % lx, j = jlo + (q / lx) % ly, k = klo + q / (lx * ly);
    const int n = i + gr.nnx * (j + gr.nny * k);
    const uint8_t fb = fixed ? fixed[n] : 0;
    const T rx = hh * (T)(2 * i - ilo - ihi), ry = hh * (T)(2 * j - jlo - jhi), rz = hh * (T)(2 * k - klo - khi);
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

// Elements of a box [X0,X1]x[Y0,Y1]x[Z0,Z1] minus an inner box [x0,x1]x[y0,y1]x[z0,z1]
// (the shell), enumerated in z-layer, row, column order.
struct Shell {
  int X0, Y0, Z0, LX, LY, LZ;   // outer box origin and extent
  int x0, y0, z0, IX, IY, IZ;   // inner box origin and extent (all > 0, or none)
  int A, Rg, nlo, nmid;          // layer area, ring area, full layers below, ring layers
  int count;
  __host__ __device__ void init(int X0_, int X1, int Y0_, int Y1, int Z0_, int Z1, int x0_, int x1, int y0_, int y1,
                                int z0_, int z1, bool full) {
    X0 = X0_; Y0 = Y0_; Z0 = Z0_;
    LX = X1 - X0 + 1; LY = Y1 - Y0 + 1; LZ = Z1 - Z0 + 1;
    x0 = x0_; y0 = y0_; z0 = z0_;
    IX = x1 - x0 + 1 > 0 ? x1 - x0 + 1 : 0;
    IY = y1 - y0 + 1 > 0 ? y1 - y0 + 1 : 0;
    IZ = z1 - z0 + 1 > 0 ? z1 - z0 + 1 : 0;
    if (full || IX == 0 || IY == 0 || IZ == 0) { IX = IY = IZ = 0; x0 = X0; y0 = Y0; z0 = Z0; }
    A = LX * LY;
    Rg = A - IX * IY;
    nlo = IZ ? (z0 - Z0) : LZ;
    nmid = IZ;
    count = (LX > 0 && LY > 0 && LZ > 0) ? (LZ - IZ) * A + IZ * Rg : 0;
  }
  __device__ void at(int q, int& x, int& y, int& z) const {
    if (q < nlo * A) {
      z = Z0 + q / A;
      const int t = q % A;
      x = X0 + t % LX;
      y = Y0 + t / LX;
      return;
    }
    q -= nlo * A;
    if (q < nmid * Rg) {
      z = z0 + q / Rg;
      int u = q % Rg;
      const int nb = (y0 - Y0) * LX;
      if (u < nb) {
        y = Y0 + u / LX;
        x = X0 + u % LX;
        return;
      }
      u -= nb;
      const int side = LX - IX;
      if (u < IY * side) {
        y = y0 + u / side;
        const int c = u % side, left = x0 - X0;
        x = c < left ? X0 + c : x0 + IX + (c - left);
        return;
      }
      u -= IY * side;
      y = y0 + IY + u / LX;
      x = X0 + u % LX;
      return;
    }
    q -= nmid * Rg;
    z = z0 + IZ + q / A;
    const int t = q % A;
    x = X0 + t % LX;
    y = Y0 + t / LX;
  }
};

// Node shell of group G: the nodes where (K W_G) can be nonzero.  K W_G
// vanishes at a node all of whose elements lie inside G and hold no fixed
// DOF (the rigid motions are in the null space of the element stiffness), so
// the shell is the box [lo-1, hi+1]^3 (clipped to the grid) minus an inner
// box inside [lo+1, hi-1]^3.  When G holds fixed nodes (bounding box fb =
// {imin, imax, jmin, jmax, kmin, kmax}, or fb[1] < fb[0] for none), every
// element touching one lies within fb dilated by one node, so the inner box
// is cut back on the one side (axis and direction) that keeps it largest
// while clear of that dilated box; an empty inner box leaves the whole box.
// b[0..5] outer box, b[6..11] inner box (empty when an extent is < 1).
__host__ __device__ inline void node_shell_bounds(const Grid& gr, const Groups& gp, int G, const int* fb,
                                                  int (&b)[12]) {
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  const int X[3] = {Gx, Gy, Gz}, NG[3] = {gp.ngx, gp.ngy, gp.ngz}, N[3] = {gr.nx, gr.ny, gr.nz};
  for (int d = 0; d < 3; ++d) {
    const int lo = gp.g * X[d], hi = (X[d] == NG[d] - 1) ? N[d] : gp.g * X[d] + gp.g - 1;
    b[2 * d] = lo > 0 ? lo - 1 : 0;          // outer box
    b[2 * d + 1] = hi < N[d] ? hi + 1 : N[d];
    b[6 + 2 * d] = lo + 1;                   // inner box
    b[6 + 2 * d + 1] = hi - 1;
  }
  if (!fb || fb[1] < fb[0]) return;
  int D[6];
  bool inter = true;
  for (int d = 0; d < 3; ++d) {
    D[2 * d] = fb[2 * d] - 1;
    D[2 * d + 1] = fb[2 * d + 1] + 1;
    inter = inter && D[2 * d] <= b[6 + 2 * d + 1] && D[2 * d + 1] >= b[6 + 2 * d];
  }
  if (!inter) return;
  long long best = 0;
  int blo = 0, bhi = -1, bd = 0;
  for (int d = 0; d < 3; ++d) {
    for (int side = 0; side < 2; ++side) {
      int lo = b[6 + 2 * d], hi = b[6 + 2 * d + 1];
      if (side == 0)
        lo = lo > D[2 * d + 1] + 1 ? lo : D[2 * d + 1] + 1;
      else
        hi = hi < D[2 * d] - 1 ? hi : D[2 * d] - 1;
      long long vol = hi >= lo ? (long long)(hi - lo + 1) : 0;
      for (int e = 0; e < 3; ++e)
        if (e != d) {
          const int ext = b[6 + 2 * e + 1] - b[6 + 2 * e] + 1;
          vol *= ext > 0 ? ext : 0;
        }
      if (vol > best) {
        best = vol;
        blo = lo;
        bhi = hi;
        bd = d;
      }
    }
  }
  if (best > 0) {
    b[6 + 2 * bd] = blo;
    b[6 + 2 * bd + 1] = bhi;
  } else {
    b[7] = b[6] - 1;   // no inner box: the whole box
  }
}

__host__ __device__ inline int node_shell_count(const Grid& gr, const Groups& gp, int G, const int* fb) {
  int b[12];
  node_shell_bounds(gr, gp, G, fb, b);
  const int LX = b[1] - b[0] + 1, LY = b[3] - b[2] + 1, LZ = b[5] - b[4] + 1;
  int IX = b[7] - b[6] + 1, IY = b[9] - b[8] + 1, IZ = b[11] - b[10] + 1;
  if (IX <= 0 || IY <= 0 || IZ <= 0) IX = IY = IZ = 0;
  return LX * LY * LZ - IX * IY * IZ;
}

// K W_G on the node shell of every group, stored per group as 18 arrays
// (mode m, component c) over the shell slots: AW[off_G + (6c + m) * n_G + q]
// = (K W_G)_{(node q, c), m}.  Gathered per slot from its (up to) eight
// elements in a fixed order (deterministic); element math in TC.  Elements
// whose nodes all lie in G with no fixed DOF contribute nothing.  One block
// per (group, split).
template <typename TC>
__global__ void __launch_bounds__(128)
k_build_aw(Grid gr, Groups gp, int nsplit, const double* __restrict__ Emod, const uint8_t* __restrict__ fixed,
           const int* __restrict__ gbox, const long long* __restrict__ aw_off, ElemConsts<TC> K, TC* __restrict__ AW,
           int* __restrict__ aw_node) {
  const int G = blockIdx.x, sp = blockIdx.y;
  int b[12];
  node_shell_bounds(gr, gp, G, gbox ? gbox + 6 * G : nullptr, b);
  Shell sh;
  sh.init(b[0], b[1], b[2], b[3], b[4], b[5], b[6], b[7], b[8], b[9], b[10], b[11], false);
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  int ilo, ihi, jlo, jhi, klo, khi;
  group_range(Gx, gp.g, gp.ngx, gr.nx, ilo, ihi);
  group_range(Gy, gp.g, gp.ngy, gr.ny, jlo, jhi);
  group_range(Gz, gp.g, gp.ngz, gr.nz, klo, khi);
  const TC hh = (TC)(0.5 * gp.h);
  const int nG = sh.count;
  TC* out = AW + aw_off[G];
  const int per = (nG + nsplit - 1) / nsplit;
  const int qb = sp * per, qe = min(qb + per, nG);
  for (int q = qb + threadIdx.x; q < qe; q += blockDim.x) {
    int ni, nj, nk;
    sh.at(q, ni, nj, nk);
    TC acc[18];
#pragma unroll
    for (int t = 0; t < 18; ++t) acc[t] = TC(0);
    const uint8_t fbn = fixed ? fixed[ni + gr.nnx * (nj + gr.nny * nk)] : 0;
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
      const int ei = ni - 1 + (d & 1), ej = nj - 1 + ((d >> 1) & 1), ek = nk - 1 + ((d >> 2) & 1);
      if (ei < 0 || ei >= gr.nx || ej < 0 || ej >= gr.ny || ek < 0 || ek >= gr.nz) continue;
      const int la = (1 - (d & 1)) + 2 * (1 - ((d >> 1) & 1)) + 4 * (1 - ((d >> 2) & 1));  // node q in e
      bool inG[8];
      uint8_t fb[8];
      bool anyG = false, leaves = false, anyfix = false;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int i = ei + (a & 1), j = ej + ((a >> 1) & 1), k = ek + ((a >> 2) & 1);
        inG[a] = i >= ilo && i <= ihi && j >= jlo && j <= jhi && k >= klo && k <= khi;
        fb[a] = fixed ? fixed[i + gr.nnx * (j + gr.nny * k)] : 0;
        anyG |= inG[a];
        leaves |= !inG[a];
        anyfix |= fb[a] != 0;
      }
      if (!anyG || (!leaves && !anyfix)) continue;
      const TC Ee = (TC)Emod[ei + gr.nx * (ej + gr.ny * ek)];
#pragma unroll 1
      for (int col = 0; col < 6; ++col) {
        TC v[3][8];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int i = ei + (a & 1), j = ej + ((a >> 1) & 1), k = ek + ((a >> 2) & 1);
          const TC rx = hh * (TC)(2 * i - ilo - ihi), ry = hh * (TC)(2 * j - jlo - jhi), rz = hh * (TC)(2 * k - klo - khi);
          TC w0 = 0, w1 = 0, w2 = 0;
          if (col == 0) w0 = 1;
          else if (col == 1) w1 = 1;
          else if (col == 2) w2 = 1;
          else if (col == 3) { w1 = -rz; w2 = ry; }
          else if (col == 4) { w0 = rz; w2 = -rx; }
          else { w0 = -ry; w1 = rx; }
          v[0][a] = (inG[a] && !(fb[a] & 1)) ? w0 : TC(0);
          v[1][a] = (inG[a] && !(fb[a] & 2)) ? w1 : TC(0);
          v[2][a] = (inG[a] && !(fb[a] & 4)) ? w2 : TC(0);
        }
        hex8_apply(v, Ee, K);
        // row of node q (local index la), masked at its fixed DOFs
        TC y0 = TC(0), y1 = TC(0), y2 = TC(0);
#pragma unroll
        for (int a = 0; a < 8; ++a)
          if (a == la) { y0 = v[0][a]; y1 = v[1][a]; y2 = v[2][a]; }
        acc[0 * 6 + col] += (fbn & 1) ? TC(0) : y0;
        acc[1 * 6 + col] += (fbn & 2) ? TC(0) : y1;
        acc[2 * 6 + col] += (fbn & 4) ? TC(0) : y2;
      }
    }
#pragma unroll
    for (int t = 0; t < 18; ++t) out[(size_t)t * nG + q] = acc[t];
    aw_node[aw_off[G] / 18 + q] = ni + gr.nnx * (nj + gr.nny * nk);
  }
}

// Vector width of the flat update: 16-byte loads.
template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

// alpha = rho / p.q, with p.q summed by every block from the stencil's
// per-CTA partials in the same fixed order (st_nparts = 0: alpha = 0, the
// initial step); then x += alpha p; r -= alpha q; z = r * invd (invd per DOF,
// zero on fixed DOFs); partial sums of r.z and r.r per block.  A p.q that is
// not positive and finite stops the RHS (status -3 / -5, set by block 0).  Flat over the DOFs of each RHS with
// 16-byte vector accesses (the RHS stride vs keeps every RHS aligned).
template <typename T>
__global__ void __launch_bounds__(RED_THREADS, RED_BLOCKS / 152)
k_update(int ndof, int vs, T* __restrict__ x, T* __restrict__ r, T* __restrict__ z, const T* __restrict__ p,
         const T* __restrict__ q, const T* __restrict__ invd, double* partials, CGState* st,
         const double* __restrict__ st_parts, int st_nparts, int* done_flags) {
  using V = typename Vec<T>::type;
  constexpr int NV = Vec<T>::n;
  __shared__ double red[64];
  pdl_acquire();
  const int rhs = blockIdx.y;
  if (st[rhs].done) return;
  const size_t off = (size_t)rhs * vs;
  const int nvec = ndof / NV;
  V* xv = (V*)(x + off);
  V* rv = (V*)(r + off);
  V* zv = (V*)(z + off);
  const V* pv = (const V*)(p + off);
  const V* qv = (const V*)(q + off);
  const V* dv = (const V*)invd;
  // The first vectors of this thread and r.z are loaded before alpha is
  // formed, and each pass of the loop loads the next pass's vectors before it
  // computes its own: the kernel streams 32 bytes per DOF mostly from L2, and
  // its time is a chain of load latencies unless loads stay in flight.
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const double rz_cur = st[rhs].rz;
  V cx, cr, cp, cq, cd;
  if (t0 < nvec) {
    cx = xv[t0];
    cr = rv[t0];
    cp = pv[t0];
    cq = qv[t0];
    cd = dv[t0];
  }
  double alpha_d = 0.0;
  if (st_nparts > 0) {
    const double pap = sum_partials(st_parts + (size_t)rhs * st_nparts, st_nparts, 1, 0);
    if (!(pap > 0.0) || !isfinite(pap)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        st[rhs].status = isfinite(pap) ? -3 : -5;
        st[rhs].done = 1;
        if (done_flags) done_flags[rhs] = 1;
      }
      return;
    }
    alpha_d = rz_cur / pap;
    if (blockIdx.x == 0 && threadIdx.x == 0) st[rhs].alpha = alpha_d;
  }
  const T alpha = (T)alpha_d;
  T s[2] = {T(0), T(0)};
  for (int t = t0; t < nvec; t += stride) {
    const int tn = t + stride;
    V nx, nr, np, nq, nd;
    if (tn < nvec) {
      nx = xv[tn];
      nr = rv[tn];
      np = pv[tn];
      nq = qv[tn];
      nd = dv[tn];
    }
    T* xs = (T*)&cx;
    T* rs = (T*)&cr;
    const T* ps = (const T*)&cp;
    const T* qs = (const T*)&cq;
    const T* ds = (const T*)&cd;
    V zz;
    T* zs = (T*)&zz;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      xs[c] = fma(alpha, ps[c], xs[c]);
      rs[c] = fma(-alpha, qs[c], rs[c]);
      zs[c] = rs[c] * ds[c];
      s[0] += rs[c] * zs[c];
      s[1] += rs[c] * rs[c];
    }
    xv[t] = cx;
    rv[t] = cr;
    zv[t] = zz;
    cx = nx;
    cr = nr;
    cp = np;
    cq = nq;
    cd = nd;
  }
  // tail DOFs
  for (int d = nvec * NV + blockIdx.x * blockDim.x + threadIdx.x; d < ndof; d += gridDim.x * blockDim.x) {
    const size_t i = off + d;
    x[i] = fma(alpha, p[i], x[i]);
    const T rn = fma(-alpha, q[i], r[i]);
    r[i] = rn;
    const T zn = rn * invd[d];
    z[i] = zn;
    s[0] += rn * zn;
    s[1] += rn * rn;
  }
  pdl_release();
  double o[2];
  block_sum_to_f64<2>(s, red, o);
  if (threadIdx.x == 0) {
    partials[((size_t)rhs * gridDim.x + blockIdx.x) * 2 + 0] = o[0];
    partials[((size_t)rhs * gridDim.x + blockIdx.x) * 2 + 1] = o[1];
  }
}

// (W^T r) sums of the nodes of group G in the node planes [kb, ke): each
// thread takes node columns (i, j) of a 16-wide layout and marches along z, so
// the node index advances by a plane stride and no division is needed.
// Adds (sum r, sum (x - c) x r) into s[0..5]; r is zero on fixed DOFs.
template <typename T, typename LDF>
__device__ __forceinline__ void group_wtr_planes(const Grid& gr, const T* r, size_t off, int ilo, int ihi, int jlo,
                                                 int jhi, int klo, int khi, int kb, int ke, T hh, T (&s)[12],
                                                 LDF ld) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4, nty = blockDim.x >> 4;
  const size_t plane = (size_t)gr.nnx * gr.nny;
  for (int j = jlo + ty; j <= jhi; j += nty) {
    const T ry = hh * (T)(2 * j - jlo - jhi);
    for (int i = ilo + tx; i <= ihi; i += 16) {
      const T rx = hh * (T)(2 * i - ilo - ihi);
      const T* rp = r + off + 3 * ((size_t)i + (size_t)gr.nnx * j + plane * kb);
      T rz = hh * (T)(2 * kb - klo - khi);
      const T dz = hh * T(2);
#pragma unroll 4
      for (int k = kb; k < ke; ++k, rp += 3 * plane, rz += dz) {
        const T r0 = ld(rp), r1 = ld(rp + 1), r2 = ld(rp + 2);
        s[0] += r0;
        s[1] += r1;
        s[2] += r2;
        s[3] += ry * r2 - rz * r1;
        s[4] += rz * r0 - rx * r2;
        s[5] += rx * r1 - ry * r0;
      }
    }
  }
}

// Right-hand side of the coarse solve of the two-level preconditioner,
//   v_G = (W^T r)_G - (W^T K z)_G,   (W^T K z)_G = (K W_G)^T z,
// per (group, split, rhs): W^T r over the group's nodes, (K W_G)^T z over
// its node shell from the stored AW (slot -> node index in aw_node).  r and z
// are zero on fixed DOFs.  The group's last split block adds the nsplit
// records in order into rec[rhs][G][0..11] = (W^T r (6), v (6)).
template <typename T>
__global__ void __launch_bounds__(256)
k_coarse_rhs(Grid gr, Groups gp, int nsplit, const T* __restrict__ r, const T* __restrict__ z,
             const long long* __restrict__ aw_off, const int* __restrict__ aw_node, const T* __restrict__ AW,
             double* __restrict__ part, double* __restrict__ rec, unsigned int* __restrict__ gcount, const CGState* st) {
  __shared__ double red[32 * 12];
  pdl_acquire();
  __shared__ bool s_last;
  const int G = blockIdx.x, sp = blockIdx.y, rhs = blockIdx.z;
  if (st[rhs].done) return;
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  int ilo, ihi, jlo, jhi, klo, khi;
  group_range(Gx, gp.g, gp.ngx, gr.nx, ilo, ihi);
  group_range(Gy, gp.g, gp.ngy, gr.ny, jlo, jhi);
  group_range(Gz, gp.g, gp.ngz, gr.nz, klo, khi);
  const T hh = (T)(0.5 * gp.h);
  const size_t off = (size_t)rhs * gr.vs;
  T s[12];
#pragma unroll
  for (int t = 0; t < 12; ++t) s[t] = T(0);
  {
    const int lz = khi - klo + 1;
    const int kper = (lz + nsplit - 1) / nsplit;
    const int kb = klo + sp * kper, ke = min(kb + kper, khi + 1);
    group_wtr_planes(gr, r, off, ilo, ihi, jlo, jhi, klo, khi, kb, ke, hh, s, [](const T* p) { return __ldg(p); });
  }
  {
    const long long base = aw_off[G];
    const int nG = (int)((aw_off[G + 1] - base) / 18);
    const T* aw = AW + base;
    const int* nodes = aw_node + base / 18;
    const int per = (nG + nsplit - 1) / nsplit;
    const int qb = sp * per, qe = min(qb + per, nG);
    for (int t = qb + threadIdx.x; t < qe; t += blockDim.x) {
      const size_t d = off + 3 * (size_t)nodes[t];
      const T z0 = z[d], z1 = z[d + 1], z2 = z[d + 2];
#pragma unroll
      for (int m = 0; m < 6; ++m)
        s[6 + m] += aw[(size_t)m * nG + t] * z0 + aw[(size_t)(6 + m) * nG + t] * z1 + aw[(size_t)(12 + m) * nG + t] * z2;
    }
  }
  pdl_release();
  double o[12];
  block_sum_to_f64<12>(s, red, o);
  double* mine = part + (((size_t)rhs * gp.ng + G) * nsplit + sp) * 12;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      mine[m] = o[m];
      mine[6 + m] = o[m] - o[6 + m];
    }
    __threadfence();
    s_last = atomicAdd(&gcount[(size_t)rhs * gp.ng + G], 1u) == (unsigned)nsplit - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 12) {
    const double* pp = part + (((size_t)rhs * gp.ng + G) * nsplit) * 12;
    double v = 0.0;
    for (int s2 = 0; s2 < nsplit; ++s2) v += pp[s2 * 12 + threadIdx.x];
    rec[((size_t)rhs * gp.ng + G) * 12 + threadIdx.x] = v;
  }
  if (threadIdx.x == 0) gcount[(size_t)rhs * gp.ng + G] = 0u;
}

// Element shell of group G: the elements on which W_G (zero outside G and on
// fixed DOFs) is not a rigid motion, so that their K_e W_G,e can be nonzero:
// the elements touching G's nodes ([lo-1, hi] per axis, clipped) minus an
// inner box of elements with all eight nodes in G ([lo, hi-1]).  When G holds
// fixed nodes (bounding box fb, max < min for none) the inner box is cut back
// on the one side that keeps it largest while clear of the elements touching
// one ([fb_lo-1, fb_hi] per axis); an empty inner box leaves the whole box.
// b[0..5] outer box, b[6..11] inner box (empty when an extent is < 1).
__host__ __device__ inline void elem_shell_bounds(const Grid& gr, const Groups& gp, int G, const int* fb,
                                                  int (&b)[12]) {
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  const int X[3] = {Gx, Gy, Gz}, NG[3] = {gp.ngx, gp.ngy, gp.ngz}, N[3] = {gr.nx, gr.ny, gr.nz};
  for (int d = 0; d < 3; ++d) {
    const int lo = gp.g * X[d], hi = (X[d] == NG[d] - 1) ? N[d] : gp.g * X[d] + gp.g - 1;
    b[2 * d] = lo > 0 ? lo - 1 : 0;
    b[2 * d + 1] = hi < N[d] - 1 ? hi : N[d] - 1;
    b[6 + 2 * d] = lo;
    b[6 + 2 * d + 1] = hi - 1;
  }
  if (!fb || fb[1] < fb[0]) return;
  int D[6];
  bool inter = true;
  for (int d = 0; d < 3; ++d) {
    D[2 * d] = fb[2 * d] - 1;
    D[2 * d + 1] = fb[2 * d + 1];
    inter = inter && D[2 * d] <= b[6 + 2 * d + 1] && D[2 * d + 1] >= b[6 + 2 * d];
  }
  if (!inter) return;
  long long best = 0;
  int blo = 0, bhi = -1, bd = 0;
  for (int d = 0; d < 3; ++d) {
    for (int side = 0; side < 2; ++side) {
      int lo = b[6 + 2 * d], hi = b[6 + 2 * d + 1];
      if (side == 0)
        lo = lo > D[2 * d + 1] + 1 ? lo : D[2 * d + 1] + 1;
      else
        hi = hi < D[2 * d] - 1 ? hi : D[2 * d] - 1;
      long long vol = hi >= lo ? (long long)(hi - lo + 1) : 0;
      for (int e = 0; e < 3; ++e)
        if (e != d) {
          const int ext = b[6 + 2 * e + 1] - b[6 + 2 * e] + 1;
          vol *= ext > 0 ? ext : 0;
        }
      if (vol > best) {
        best = vol;
        blo = lo;
        bhi = hi;
        bd = d;
      }
    }
  }
  if (best > 0) {
    b[6 + 2 * bd] = blo;
    b[6 + 2 * bd + 1] = bhi;
  } else {
    b[7] = b[6] - 1;
  }
}

// Right-hand side of the coarse solve without stored K W: per (group,
// share, rhs), v_G = (W^T r)_G - (W^T K z)_G with
//   (W^T K z)_G = sum over the group's element shell of W_G,e^T (E_e K0 z_e),
// each element's forces applied in the modal form (hex8_apply) and restricted
// to its nodes in G, masked at fixed DOFs (elements inside G without fixed
// DOFs contribute nothing: the rigid motions are in the element null space).
// Records and the last-block combination as in k_coarse_rhs.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)   // FP32: 4 blocks per SM
k_coarse_rhs_cut(Grid gr, Groups gp, int nsplit, const T* __restrict__ r, const T* __restrict__ z,
                 const T* __restrict__ Emod, const uint8_t* __restrict__ fixed, const int* __restrict__ gbox,
                 ElemConsts<T> K, double* __restrict__ part, double* __restrict__ rec,
                 unsigned int* __restrict__ gcount, const CGState* st, const uint4* __restrict__ cut,
                 const long long* __restrict__ cut_off) {
  __shared__ double red[32 * 12];
  __shared__ bool s_last;
  pdl_acquire();
  const int G = blockIdx.x, sp = blockIdx.y, rhs = blockIdx.z;
  if (st[rhs].done) return;
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  int ilo, ihi, jlo, jhi, klo, khi;
  group_range(Gx, gp.g, gp.ngx, gr.nx, ilo, ihi);
  group_range(Gy, gp.g, gp.ngy, gr.ny, jlo, jhi);
  group_range(Gz, gp.g, gp.ngz, gr.nz, klo, khi);
  const T hh = (T)(0.5 * gp.h);
  const size_t off = (size_t)rhs * gr.vs;
  T s[12];
#pragma unroll
  for (int t = 0; t < 12; ++t) s[t] = T(0);
  {
    const int lz = khi - klo + 1;
    const int kper = (lz + nsplit - 1) / nsplit;
    const int kb = klo + sp * kper, ke = min(kb + kper, khi + 1);
    group_wtr_planes(gr, r, off, ilo, ihi, jlo, jhi, klo, khi, kb, ke, hh, s, [](const T* p) { return __ldg(p); });
  }
  if (cut) {
    // the group's cut elements from their records (k_build_cut_recs)
    const long long base = cut_off[G];
    const int cnt = (int)(cut_off[G + 1] - base);
    const int per = (cnt + nsplit - 1) / nsplit;
    const int qb = sp * per, qe = min(qb + per, cnt);
    const int plane = gr.nnx * gr.nny;
    const T h2 = hh + hh;
    const T bx0 = hh * (T)(ilo - ihi - 2), by0 = hh * (T)(jlo - jhi - 2), bz0 = hh * (T)(klo - khi - 2);
    for (int t = qb + threadIdx.x; t < qe; t += blockDim.x) {
      const uint4 q = __ldg(cut + base + t);
      const int n0 = (int)q.x;
      const unsigned ingrp = q.w >> 24, fbits = q.w & 0xFFFFFFu;
      T v[3][8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int n = n0 + (a & 1) + ((a >> 1) & 1) * gr.nnx + ((a >> 2) & 1) * plane;
        const T* zp = z + off + 3 * (size_t)n;
        v[0][a] = __ldg(zp);
        v[1][a] = __ldg(zp + 1);
        v[2][a] = __ldg(zp + 2);
      }
      hex8_apply(v, __ldg(Emod + q.y), K);
      // moment arms about the group centre: hh (2 i - ilo - ihi) with i = ilo - 1 + rel_i + (a & 1)
      const T bx = bx0 + h2 * (T)(int)(q.z & 1023u), by = by0 + h2 * (T)(int)((q.z >> 10) & 1023u),
              bz = bz0 + h2 * (T)(int)((q.z >> 20) & 1023u);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        if (!((ingrp >> a) & 1u)) continue;
        const unsigned fb = (fbits >> (3 * a)) & 7u;
        const T y0 = (fb & 1) ? T(0) : v[0][a];
        const T y1 = (fb & 2) ? T(0) : v[1][a];
        const T y2 = (fb & 4) ? T(0) : v[2][a];
        const T rx = (a & 1) ? bx + h2 : bx, ry = ((a >> 1) & 1) ? by + h2 : by, rz = ((a >> 2) & 1) ? bz + h2 : bz;
        s[6] += y0;
        s[7] += y1;
        s[8] += y2;
        s[9] += ry * y2 - rz * y1;
        s[10] += rz * y0 - rx * y2;
        s[11] += rx * y1 - ry * y0;
      }
    }
  } else {
    int b[12];
    elem_shell_bounds(gr, gp, G, gbox ? gbox + 6 * G : nullptr, b);
    Shell sh;
    sh.init(b[0], b[1], b[2], b[3], b[4], b[5], b[6], b[7], b[8], b[9], b[10], b[11], false);
    const int per = (sh.count + nsplit - 1) / nsplit;
    const int qb = sp * per, qe = min(qb + per, sh.count);
    for (int t = qb + threadIdx.x; t < qe; t += blockDim.x) {
      int ei, ej, ek;
      sh.at(t, ei, ej, ek);
      T v[3][8];
      uint8_t fb[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int i = ei + (a & 1), j = ej + ((a >> 1) & 1), k = ek + ((a >> 2) & 1);
        const int n = i + gr.nnx * (j + gr.nny * k);
        fb[a] = fixed ? __ldg(fixed + n) : 0;
        const T* zp = z + off + 3 * (size_t)n;
        v[0][a] = __ldg(zp);
        v[1][a] = __ldg(zp + 1);
        v[2][a] = __ldg(zp + 2);
      }
      hex8_apply(v, __ldg(Emod + ei + gr.nx * (ej + gr.ny * ek)), K);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int i = ei + (a & 1), j = ej + ((a >> 1) & 1), k = ek + ((a >> 2) & 1);
        if (i < ilo || i > ihi || j < jlo || j > jhi || k < klo || k > khi) continue;
        const T y0 = (fb[a] & 1) ? T(0) : v[0][a];
        const T y1 = (fb[a] & 2) ? T(0) : v[1][a];
        const T y2 = (fb[a] & 4) ? T(0) : v[2][a];
        const T rx = hh * (T)(2 * i - ilo - ihi), ry = hh * (T)(2 * j - jlo - jhi), rz = hh * (T)(2 * k - klo - khi);
        s[6] += y0;
        s[7] += y1;
        s[8] += y2;
        s[9] += ry * y2 - rz * y1;
        s[10] += rz * y0 - rx * y2;
        s[11] += rx * y1 - ry * y0;
      }
    }
  }
  pdl_release();
  double o[12];
  block_sum_to_f64<12>(s, red, o);
  double* mine = part + (((size_t)rhs * gp.ng + G) * nsplit + sp) * 12;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      mine[m] = o[m];
      mine[6 + m] = o[m] - o[6 + m];
    }
    __threadfence();
    s_last = atomicAdd(&gcount[(size_t)rhs * gp.ng + G], 1u) == (unsigned)nsplit - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 12) {
    const double* pp = part + (((size_t)rhs * gp.ng + G) * nsplit) * 12;
    double v = 0.0;
    for (int s2 = 0; s2 < nsplit; ++s2) v += pp[s2 * 12 + threadIdx.x];
    rec[((size_t)rhs * gp.ng + G) * 12 + threadIdx.x] = v;
  }
  if (threadIdx.x == 0) gcount[(size_t)rhs * gp.ng + G] = 0u;
}

// Records of the cut elements of every group (the shells of
// k_coarse_rhs_cut, in the same order), one block per group, written once per
// set of supports: x = node index of the element's corner (i, j, k),
// y = element index, z = the element's position relative to the group,
// (i - ilo + 1) | (j - jlo + 1) << 10 | (k - klo + 1) << 20, w = the fixed-DOF
// bits of its 8 nodes (3 per node, node a at bit 3a) | the mask of its nodes
// in the group << 24.  Needs groups at most 1022 elements wide.
__global__ void k_build_cut_recs(Grid gr, Groups gp, const uint8_t* __restrict__ fixed, const int* __restrict__ gbox,
                                 const long long* __restrict__ cut_off, uint4* __restrict__ cut) {
  const int G = blockIdx.x;
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  int ilo, ihi, jlo, jhi, klo, khi;
  group_range(Gx, gp.g, gp.ngx, gr.nx, ilo, ihi);
  group_range(Gy, gp.g, gp.ngy, gr.ny, jlo, jhi);
  group_range(Gz, gp.g, gp.ngz, gr.nz, klo, khi);
  int b[12];
  elem_shell_bounds(gr, gp, G, gbox ? gbox + 6 * G : nullptr, b);
  Shell sh;
  sh.init(b[0], b[1], b[2], b[3], b[4], b[5], b[6], b[7], b[8], b[9], b[10], b[11], false);
  const long long base = cut_off[G];
  for (int t = threadIdx.x; t < sh.count; t += blockDim.x) {
    int ei, ej, ek;
    sh.at(t, ei, ej, ek);
    unsigned fb = 0, in = 0;
    for (int a = 0; a < 8; ++a) {
      const int i = ei + (a & 1), j = ej + ((a >> 1) & 1), k = ek + ((a >> 2) & 1);
      const int n = i + gr.nnx * (j + gr.nny * k);
      fb |= (unsigned)(fixed ? fixed[n] & 7 : 0) << (3 * a);
      if (i >= ilo && i <= ihi && j >= jlo && j <= jhi && k >= klo && k <= khi) in |= 1u << a;
    }
    uint4 q;
    q.x = (unsigned)(ei + gr.nnx * (ej + gr.nny * ek));
    q.y = (unsigned)(ei + gr.nx * (ej + gr.ny * ek));
    q.z = (unsigned)(ei - ilo + 1) | (unsigned)(ej - jlo + 1) << 10 | (unsigned)(ek - klo + 1) << 20;
    q.w = fb | in << 24;
    cut[base + t] = q;
  }
}

// gbox[6G..6G+5] = bounding box (imin, imax, jmin, jmax, kmin, kmax) of the
// nodes of group G with a fixed DOF; initialised to (INT_MAX, -1, ...) so that
// an empty box has max < min.
__global__ void k_group_fixed(Grid gr, Groups gp, const uint8_t* __restrict__ fixed, int* __restrict__ gbox) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < gr.nnodes; n += gridDim.x * blockDim.x) {
    if (!fixed[n]) continue;
    const int i = n % gr.nnx, j = (n / gr.nnx) % gr.nny, k = n / (gr.nnx * gr.nny);
    const int G = group_of_axis(i, gp.g, gp.ngx) + gp.ngx * (group_of_axis(j, gp.g, gp.ngy) + gp.ngy * group_of_axis(k, gp.g, gp.ngz));
    int* bx = gbox + 6 * G;
    atomicMin(bx + 0, i); atomicMax(bx + 1, i);
    atomicMin(bx + 2, j); atomicMax(bx + 3, j);
    atomicMin(bx + 4, k); atomicMax(bx + 5, k);
  }
}

__global__ void k_group_box_init(int ng, int* __restrict__ gbox) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 6 * ng; t += gridDim.x * blockDim.x)
    gbox[t] = (t & 1) ? -1 : 0x7fffffff;
}

// W mu at node (i, j, k): t + omega x r of the node's group (zero on fixed DOFs).
template <typename T>
__device__ __forceinline__ void prolong_node(const Grid& gr, const Groups& gp, const double* mu, int i, int j, int k,
                                             T (&w)[3]) {
  const int Gx = group_of_axis(i, gp.g, gp.ngx), Gy = group_of_axis(j, gp.g, gp.ngy), Gz = group_of_axis(k, gp.g, gp.ngz);
  const int G = Gx + gp.ngx * (Gy + gp.ngy * Gz);
  const double* m = mu + 6 * G;
  int lo, hi;
  const T hh = (T)(0.5 * gp.h);
  group_range(Gx, gp.g, gp.ngx, gr.nx, lo, hi);
  const T rx = hh * (T)(2 * i - lo - hi);
  group_range(Gy, gp.g, gp.ngy, gr.ny, lo, hi);
  const T ry = hh * (T)(2 * j - lo - hi);
  group_range(Gz, gp.g, gp.ngz, gr.nz, lo, hi);
  const T rz = hh * (T)(2 * k - lo - hi);
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
  const size_t off = (size_t)rhs * gr.vs;
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

// Coarse solve mu[rhs] = Einv v[rhs] (Einv symmetric, row-major, type TE);
// one warp per row, all RHS (used by the deflated start).
template <typename TE>
__global__ void __launch_bounds__(256)
k_coarse_solve(int nc, int nrhs, const TE* __restrict__ Einv, const double* __restrict__ v, double* __restrict__ mu,
               const CGState* st) {
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= nc) return;
  const TE* er = Einv + (size_t)row * nc;
  for (int r = 0; r < nrhs; ++r) {
    if (st && st[r].done) continue;
    const double* vr = v + (size_t)r * nc;
    TE s = TE(0);
    for (int c = lane; c < nc; c += 32) s = fma(er[c], (TE)vr[c], s);
    s = warp_sum(s);
    if (lane == 0) mu[(size_t)r * nc + row] = (double)s;
  }
}

// One row of the dense coarse inverse times v (staged in shared memory in the
// row's own type), by one warp.  The row is read as 16-byte vectors when its
// length allows, in batches of 8 vectors per lane whose loads are all issued
// before any is consumed: a row of n_c = 768 FP32 values is one memory round
// trip instead of a chain of dependent ones.
template <typename TE> struct Vec16;
template <> struct Vec16<float> { using T = float4; static constexpr int N = 4; };
template <> struct Vec16<double> { using T = double2; static constexpr int N = 2; };
__device__ __forceinline__ float vdot(float4 a, float4 b, float s) {
  s = fmaf(a.x, b.x, s);
  s = fmaf(a.y, b.y, s);
  s = fmaf(a.z, b.z, s);
  return fmaf(a.w, b.w, s);
}
__device__ __forceinline__ double vdot(double2 a, double2 b, double s) {
  s = fma(a.x, b.x, s);
  return fma(a.y, b.y, s);
}
template <typename TE>
__device__ __forceinline__ TE coarse_row_dot(const TE* __restrict__ er, const TE* vt, int nc, int lane) {
  using VT = typename Vec16<TE>::T;
  constexpr int V = Vec16<TE>::N, U = 8;
  TE s = TE(0);
  if (nc % V == 0) {
    const VT* ev = reinterpret_cast<const VT*>(er);
    const VT* vv = reinterpret_cast<const VT*>(vt);
    const int nv = nc / V;
    for (int base = 0; base < nv; base += 32 * U) {
      VT e[U];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int c = base + lane + 32 * j;
        if (c < nv) e[j] = __ldg(ev + c);
      }
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int c = base + lane + 32 * j;
        if (c < nv) s = vdot(e[j], vv[c], s);
      }
    }
  } else {
    for (int c = lane; c < nc; c += 32) s = fma(er[c], vt[c], s);
  }
  return warp_sum(s);
}

// Coarse step of one DPCG iteration: v_G and (W^T r)_G are read from the
// per-group k_coarse_rhs records, mu = Einv v (one warp per row, all RHS),
// and each block leaves its rows' share of (W^T r).mu in cd_parts, from which
// rho = r.z + (W^T r).mu (the preconditioned residual y = z + W mu of the
// two-level operator) follows.  Inside the loop (fin == 1) that is all: the
// next stencil forms rho, r.r, beta and the stopping test
// (dpcg_iteration_start).  For the initial step (fin == 2) the last block to
// finish takes them here, in one pass over the k_update partials and the
// cd_parts (beta = 0), so that an initial residual already below the target
// stops before the loop.
template <typename TE>
__global__ void __launch_bounds__(256)
k_coarse_step(int nc, int nrhs, const TE* __restrict__ Einv, double* __restrict__ mu, CGState* st,
              const double* __restrict__ rec, double* __restrict__ cd_parts, int fin, int* done_flags,
              unsigned int* counter, const double* __restrict__ upd_partials, int upd_nparts,
              double* __restrict__ upd_red) {
  using VT = typename Vec16<TE>::T;
  constexpr int V = Vec16<TE>::N, U = 8;
  extern __shared__ __align__(16) double vs[];   // nc values of v for the current RHS (as TE)
  TE* vt = reinterpret_cast<TE*>(vs);
  __shared__ double wcd[32];
  __shared__ double red[32 * 3];
  __shared__ bool s_last;
  pdl_acquire();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int row = blockIdx.x * nwarps + warp;
  const int ng = nc / 6;
  // The row of the inverse does not depend on the iteration: its loads are
  // issued first, so that they overlap the loads of v and of the state (the
  // kernel is a chain of memory latencies, not bandwidth).  Rows that fit in
  // one batch of U vectors per lane stay in registers for every RHS.
  // The vector update's (r.z, r.r) partials are summed here in slices, one per
  // block in block order (each slice in index order), so that the next
  // stencil's every CTA sums gridDim.x slices instead of all of them.  This
  // block is latency-bound: the few extra loads overlap its GEMV.
  if (upd_red && threadIdx.x < 2 * nrhs) {
    const int r = threadIdx.x >> 1, comp = threadIdx.x & 1;
    const int per = (upd_nparts + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(i0 + per, upd_nparts);
    const double* up = upd_partials + (size_t)r * upd_nparts * 2;
    double sum = 0.0;
    for (int i = i0; i < i1; ++i) sum += up[2 * i + comp];
    upd_red[((size_t)r * gridDim.x + blockIdx.x) * 2 + comp] = sum;
  }
  const int nv = nc / V;
  const bool in_regs = nc % V == 0 && nv <= 32 * U;
  VT e[U];
  if (in_regs && row < nc) {
    const VT* ev = reinterpret_cast<const VT*>(Einv + (size_t)row * nc);
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int c = lane + 32 * j;
      if (c < nv) e[j] = __ldg(ev + c);
    }
  }
  for (int r = 0; r < nrhs; ++r) {
    if (st[r].done) continue;
    const double* rr = rec + (size_t)r * ng * 12;
    const double wtr = (row < nc && lane == 0) ? rr[(row / 6) * 12 + row % 6] : 0.0;
    for (int q = threadIdx.x; q < nc; q += blockDim.x) vt[q] = (TE)rr[(q / 6) * 12 + 6 + q % 6];
    __syncthreads();
    double cd = 0.0;
    if (row < nc) {
      TE s;
      if (in_regs) {
        const VT* vv = reinterpret_cast<const VT*>(vt);
        s = TE(0);
#pragma unroll
        for (int j = 0; j < U; ++j) {
          const int c = lane + 32 * j;
          if (c < nv) s = vdot(e[j], vv[c], s);
        }
        s = warp_sum(s);
      } else {
        s = coarse_row_dot<TE>(Einv + (size_t)row * nc, vt, nc, lane);
      }
      if (lane == 0) {
        mu[(size_t)r * nc + row] = (double)s;
        cd = wtr * (double)s;
      }
    }
    if (lane == 0) wcd[warp] = cd;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < nwarps; ++w) t += wcd[w];
      cd_parts[(size_t)r * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
  pdl_release();
  // fin == 1: the loop's stencil forms beta and the stopping test from the
  // cd_parts (dpcg_iteration_start); the initial step (fin == 2) takes them
  // here, in the last block, for every RHS
  if (fin == 1) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int r = 0; r < nrhs; ++r) {
    CGState& S = st[r];
    if (S.done) continue;
    // the state's fields are loaded with the partials, not after their sum
    double rz_old = 0.0, target2 = 0.0;
    int iters = 0, max_iters = 0;
    if (threadIdx.x == 0) {
      rz_old = S.rz;
      target2 = S.target2;
      iters = S.iters;
      max_iters = S.max_iters;
    }
    double ps[3] = {0.0, 0.0, 0.0};
    const double2* up = (const double2*)(upd_partials + (size_t)r * upd_nparts * 2);
    for (int i = threadIdx.x; i < upd_nparts; i += blockDim.x) {
      const double2 v = up[i];
      ps[0] += v.x;
      ps[1] += v.y;
    }
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) ps[2] += cd_parts[(size_t)r * gridDim.x + i];
    double o[3];
    block_sum_to_f64<3>(ps, red, o);
    if (threadIdx.x == 0) {
      const double rz = o[0], rr = o[1], rho = rz + o[2];
      int done = 0;
      if (!isfinite(rr) || !isfinite(rho)) {
        S.status = -5;
        done = 1;
      } else {
        S.beta = fin == 2 ? 0.0 : rho / rz_old;
        if (fin != 2) iters += 1;
        S.iters = iters;
        S.rz = rho;
        S.rr = rr;
        if (rr <= target2) {
          done = 1;
          S.status = 0;
        } else if (iters >= max_iters) {
          done = 1;
          S.status = -3;
        }
      }
      S.done = done;
      if (done_flags) done_flags[r] = done;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// ---------------------------------------------------------------------------
// Mixed-precision refinement helpers
// ---------------------------------------------------------------------------

// u64 += (double) d32  (per RHS; skip RHS whose outer loop has converged)
__global__ void k_accumulate(int ndof, int vs, double* __restrict__ u, const float* __restrict__ d, const int* skip) {
  const int rhs = blockIdx.y;
  if (skip && skip[rhs]) return;
  const size_t off = (size_t)rhs * vs;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ndof; i += gridDim.x * blockDim.x)
    u[off + i] += (double)d[off + i];
}

template <typename T>
__global__ void k_fill(size_t n, T* __restrict__ x, T v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] = v;
}

// Partial sums of x.y (FP64) per block, per RHS (n values, RHS stride vs).
template <typename T, typename U>
__global__ void __launch_bounds__(RED_THREADS)
k_dot(int n, int vs, const T* __restrict__ x, const U* __restrict__ y, double* partials) {
  __shared__ double red[32];
  const int rhs = blockIdx.y;
  const size_t off = (size_t)rhs * vs;
  double s[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s[0] = fma((double)x[off + i], (double)y[off + i], s[0]);
  double o[1];
  block_sum_to_f64<1>(s, red, o);
  if (threadIdx.x == 0) partials[(size_t)rhs * gridDim.x + blockIdx.x] = o[0];
}

}  // namespace afd

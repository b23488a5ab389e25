// Matrix-free stiffness apply y = K u on the voxel hex8 mesh (Sec. 3.5: the
// system is solved without assembling K; the cost is memory traffic).
//
// Design (sm_103a).  Every thread owns one node column (i, j) and marches
// along z; a CTA is 32 lanes (x) by TY warps (y).  The element operator is
// applied in the Walsh-Hadamard modal form of afd_common.cuh, with the three
// butterfly stages factorised across the grid instead of per element:
//   x stage: sum/difference of the node and its +x neighbour (warp shuffle),
//   y stage: sum/difference of two x-edges (one shared-memory exchange),
//   z stage: sum/difference of the face values of two planes (registers),
// so every x-edge and face is transformed once, not once per element.  The
// transposed stages run in reverse order on the element forces: the two
// elements sharing a face are added before the face is split into edges, and
// the two faces sharing an edge before it is split into nodes.  Nothing goes
// through global atomics; CTAs overlap by one column in x and one row in y so
// every node is finished by exactly one thread.
#pragma once

#include <type_traits>
#include "afd_common.cuh"
#include "dpcg_kernels.cuh"

namespace afd {

enum StencilMode {
  ST_APPLY = 0,     // y = K u
  ST_RESIDUAL = 1,  // y = f - K u, partial sum y.y, optional float copy of y
  ST_APPLY_DOT = 2,  // y = K u, partial sum u.y; u formed as the search direction (see z below)
  ST_DOT_PLAIN = 3   // y = K u, partial sum u.y, u read as given (FP32 packed kernel only)
};

template <typename T, typename TF>
struct StencilArgs {
  Grid gr;
  const T* u;             // [rhs][ndof]
  T* y;                   // [rhs][ndof] (ST_RESIDUAL: nullable, then only the norm and y32 are formed)
  const T* E;             // [nelem] element moduli in the working type
  const uint8_t* fixed;   // [nnodes] bit c set = DOF c fixed (nullable: none fixed)
  ElemConsts<T> K;
  const TF* f;            // ST_RESIDUAL: [rhs][ndof]
  float* y32;             // ST_RESIDUAL: optional float copy of y
  double* partials;       // [rhs][nblocks] (ST_RESIDUAL, ST_APPLY_DOT)
  const int* done;        // [rhs] skip the work when nonzero (nullable)
  int kz;                 // node planes per CTA
  int tiles_x;            // CTAs along x
  // ST_APPLY_DOT with a counter: the last CTA of each RHS turns the u.y
  // partials into the CG step length alpha = rho / (p.Ap) (the solver leaves
  // counter null and lets the vector update form alpha)
  CGState* st;
  unsigned int* counter;  // [rhs], zero between launches
  // Fused search-direction update (nullable z): the applied vector is
  // p = z + W mu + beta p_old, formed as each node is loaded (u holds p_old,
  // beta comes from st), and written back to pout at the nodes this CTA owns.
  const T* z;
  const double* mu;       // [rhs][6 N_g]
  T* pout;
  Groups gp;
  // ST_APPLY_DOT inside the solver loop (non-null ip.upd): beta and the
  // stopping test are formed at kernel start from the previous iteration's
  // partials (dpcg_iteration_start); otherwise beta is read from st
  IterPartials ip;
};

constexpr int ST_TX = 32;  // lanes per warp; lanes 1..30 finish nodes, lane 31 is a halo column

// Launch geometry: a CTA of TY warps finishes (ST_TX-2) x (TY-2) node columns
// over kz planes (TY-1 element rows; the last warp only supplies x-edges).
template <int TY>
struct StencilGeom {
  static void get(const Grid& gr, int kz, int& tiles_x, dim3& grid) {
    tiles_x = (gr.nnx + (ST_TX - 3)) / (ST_TX - 2);
    const int tiles_y = (gr.nny + (TY - 3)) / (TY - 2);
    const int zch = (gr.nnz + kz - 1) / kz;
    grid = dim3(tiles_x * tiles_y, zch, 1);
  }
};

// Element constants in the kernel's arithmetic type (a no-op copy when it is
// the storage type).
template <typename C, typename T>
__device__ __forceinline__ ElemConsts<C> elem_consts_as(const ElemConsts<T>& k) {
  using A = Arith<C, T>;
  ElemConsts<C> c;
  c.l16 = A::in(k.l16);
  c.m16 = A::in(k.m16);
  c.m8 = A::in(k.m8);
  c.l48 = A::in(k.l48);
  c.m48 = A::in(k.m48);
  c.m3_48 = A::in(k.m3_48);
  c.t144 = A::in(k.t144);
  return c;
}

// T: the type of u, y, z, p and E in memory; C: the arithmetic type (T, or
// dfloat for an FP64-accurate residual computed on the FP32 pipes).
template <typename T, int TY, int MODE, typename TF, typename C = T>
__global__ void __launch_bounds__(ST_TX * TY, std::is_same<C, dfloat>::value ? 2 : 1)
stencil_kernel(const StencilArgs<T, TF> a) {
  using AT = Arith<C, T>;
  const ElemConsts<C> K = elem_consts_as<C>(a.K);
  pdl_acquire();
  // TY warps: warps 0..TY-2 own element rows, the last warp only supplies the
  // x-edges of the row above the tile.  Exchange buffers: each is written,
  // then read after a barrier; the other exchange's barrier separates that
  // read from the next write.
  __shared__ C xe[6][TY][ST_TX];   // x-edge (S, D) x 3 components
  __shared__ C ye[6][TY][ST_TX];   // edge contributions sent to the row above
  __shared__ double red[32];

  const int rhs = blockIdx.z;
  if (a.done && a.done[rhs]) return;
  const Grid gr = a.gr;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tile_x = blockIdx.x % a.tiles_x;
  const int tile_y = blockIdx.x / a.tiles_x;
  const int i = tile_x * (ST_TX - 2) - 1 + lane;   // node / element column
  const int j = tile_y * (TY - 2) - 1 + w;
  const int k0 = blockIdx.y * a.kz;
  const int k1 = min(k0 + a.kz, gr.nnz);
  const size_t voff = (size_t)rhs * gr.vs;
  const T* __restrict__ u = a.u + voff;

  const bool col_ok = i >= 0 && i < gr.nnx && j >= 0 && j < gr.nny;
  const bool elem_xy = lane < ST_TX - 1 && i >= 0 && i < gr.nx && j >= 0 && j < gr.ny && w < TY - 1;
  const bool out_xy = lane >= 1 && lane < ST_TX - 1 && w >= 1 && w < TY - 1 && i <= gr.nx && j <= gr.ny;

  // Fused search direction p = z + W mu + beta p_old.  For this thread's
  // column the rigid motion of group G is W mu = A_G + r_z B_G with
  // A_G = t + omega x (r_x, r_y, 0), B_G = (omega_y, -omega_x, 0); A, B are
  // refreshed when the plane index enters the next group along z.
  const bool formp = a.z != nullptr;
  C beta = C(0);
  if (formp) {
    if (a.ip.upd) {
      double b;
      if (!dpcg_iteration_start(a.st, rhs, const_cast<int*>(a.done), a.ip, b)) return;
      beta = (C)b;
    } else {
      beta = (C)a.st[rhs].beta;
    }
  }
  const Groups gp = a.gp;
  const C hh = (C)(0.5 * gp.h);
  C rx = C(0), ry = C(0);
  int gxy = 0;            // Gx + ngx * Gy
  int gz = -1, gz_next = 0, zlo = 0, zhi = 0;
  C A0 = C(0), A1 = C(0), A2 = C(0), B0 = C(0), B1 = C(0);
  const double* murhs = formp ? a.mu + (size_t)rhs * 6 * gp.ng : nullptr;
  if (formp && col_ok) {
    int lo, hi;
    const int Gx = group_of_axis(i, gp.g, gp.ngx), Gy = group_of_axis(j, gp.g, gp.ngy);
    group_range(Gx, gp.g, gp.ngx, gr.nx, lo, hi);
    rx = hh * (C)(2 * i - lo - hi);
    group_range(Gy, gp.g, gp.ngy, gr.ny, lo, hi);
    ry = hh * (C)(2 * j - lo - hi);
    gxy = Gx + gp.ngx * Gy;
  }
  auto refresh_group = [&](int k) {
    gz = group_of_axis(k, gp.g, gp.ngz);
    group_range(gz, gp.g, gp.ngz, gr.nz, zlo, zhi);
    gz_next = (gz == gp.ngz - 1) ? (1 << 30) : zhi + 1;
    const double* m6 = murhs + 6 * (gxy + gp.ngx * gp.ngy * gz);
    const C tx = (C)m6[0], ty = (C)m6[1], tz = (C)m6[2], ox = (C)m6[3], oy = (C)m6[4], oz = (C)m6[5];
    A0 = tx - oz * ry;
    A1 = ty + oz * rx;
    A2 = tz + (ox * ry - oy * rx);
    B0 = oy;
    B1 = -ox;
  };

  auto load_node = [&](int k, C (&v)[3]) {
    if (col_ok && k >= 0 && k < gr.nnz) {
      const int n = i + gr.nnx * (j + gr.nny * k);
      const uint8_t fb = a.fixed ? a.fixed[n] : 0;
      const T* p = u + 3 * (size_t)n;
      if (formp) {
        if (k >= gz_next || gz < 0) refresh_group(k);
        const T* zz = a.z + voff + 3 * (size_t)n;
        const C rz = hh * (C)(2 * k - zlo - zhi);
        v[0] = (fb & 1) ? C(0) : fma(beta, AT::in(p[0]), AT::in(zz[0]) + fma(rz, B0, A0));
        v[1] = (fb & 2) ? C(0) : fma(beta, AT::in(p[1]), AT::in(zz[1]) + fma(rz, B1, A1));
        v[2] = (fb & 4) ? C(0) : fma(beta, AT::in(p[2]), AT::in(zz[2]) + A2);
      } else {
        v[0] = (fb & 1) ? C(0) : AT::in(p[0]);
        v[1] = (fb & 2) ? C(0) : AT::in(p[1]);
        v[2] = (fb & 4) ? C(0) : AT::in(p[2]);
      }
    } else {
      v[0] = v[1] = v[2] = C(0);
    }
  };

  // face values (x-edge stage then y stage) of a node plane for element column (i, j):
  // F[c][q], q = mx + 2 my (mx: x-difference, my: y-difference)
  auto face_values = [&](const C (&un)[3], C (&F)[3][4]) {
    C S[3], D[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const C right = __shfl_down_sync(0xffffffffu, un[c], 1);  // lane 31: unused
      S[c] = right + un[c];
      D[c] = right - un[c];
      xe[c][w][lane] = S[c];
      xe[3 + c][w][lane] = D[c];
    }
    __syncthreads();
    if (w < TY - 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const C S1 = xe[c][w + 1][lane], D1 = xe[3 + c][w + 1][lane];
        F[c][0] = S1 + S[c];
        F[c][1] = D1 + D[c];
        F[c][2] = S1 - S[c];
        F[c][3] = D1 - D[c];
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) F[c][0] = F[c][1] = F[c][2] = F[c][3] = C(0);
    }
  };

  C Fb[3][4];      // face values of the plane below the current element layer
  C Tprev[3][4];   // top-face forces of the element layer below the current plane
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) Fb[c][q] = Tprev[c][q] = C(0);

  {
    C un0[3];
    load_node(k0 - 1, un0);
    face_values(un0, Fb);
    __syncthreads();  // the loop's first x-edge write follows this read
  }
  C ucur[3] = {C(0), C(0), C(0)};   // (formed) u at (i, j, l) for the dot epilogue and p write
  C part = C(0);
  C un[3];
  load_node(k0, un);   // prefetch of the next plane

  for (int l = k0 - 1; l < k1; ++l) {
    // element layer l lies between node planes l and l+1; finish plane l
    C Ft[3][4];
    face_values(un, Ft);
    const C u_l1[3] = {un[0], un[1], un[2]};  // plane l+1
    C E = C(0);
    if (elem_xy && l >= 0 && l < gr.nz) E = AT::in(a.E[i + gr.nx * (j + gr.ny * l)]);
    if (l + 2 <= k1) load_node(l + 2, un);  // prefetch plane l+2
    C Bf[3][4];  // bottom-face forces of element layer l (plane l)
    if (E != C(0)) {
      C h[3][8];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          h[c][q] = Ft[c][q] + Fb[c][q];
          h[c][q + 4] = Ft[c][q] - Fb[c][q];
        }
      modal_forces(h, E, K);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const C g0 = h[c][q], g1 = h[c][q + 4];
          Bf[c][q] = g0 - g1;
          const C tf = g0 + g1;
          h[c][q] = tf;   // keep the top-face force
        }
      // plane l total face force: this layer's bottom + the layer below's top
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          Bf[c][q] += Tprev[c][q];
          Tprev[c][q] = h[c][q];
        }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          Bf[c][q] = Tprev[c][q];
          Tprev[c][q] = C(0);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) Fb[c][q] = Ft[c][q];

    // transposed y stage: face (i, j) -> x-edges of rows j and j+1
    C e0[3][2], e1[3][2];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int mx = 0; mx < 2; ++mx) {
        e0[c][mx] = Bf[c][mx] - Bf[c][mx + 2];
        e1[c][mx] = Bf[c][mx] + Bf[c][mx + 2];
      }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ye[2 * c][w][lane] = e1[c][0];
      ye[2 * c + 1][w][lane] = e1[c][1];
    }
    __syncthreads();
    if (w >= 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        e0[c][0] += ye[2 * c][w - 1][lane];
        e0[c][1] += ye[2 * c + 1][w - 1][lane];
      }
    }
    // transposed x stage: edge (i, i+1) -> node i gets s - d, node i+1 gets s + d
    C yv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const C sp = e0[c][0] + e0[c][1];
      const C from_left = __shfl_up_sync(0xffffffffu, sp, 1);
      yv[c] = (e0[c][0] - e0[c][1]) + (lane >= 1 ? from_left : C(0));
    }
    if (l >= k0 && out_xy) {
      const int n = i + gr.nnx * (j + gr.nny * l);
      const uint8_t fb = a.fixed ? a.fixed[n] : 0;
      T* yp = a.y ? a.y + voff + 3 * (size_t)n : nullptr;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const bool fx = (fb >> c) & 1;
        C out;
        if (MODE == ST_RESIDUAL) {
          out = fx ? C(0) : Arith<C, TF>::in(a.f[voff + 3 * (size_t)n + c]) - yv[c];
          part += out * out;
          if (a.y32) a.y32[voff + 3 * (size_t)n + c] = (float)out;
        } else {
          out = fx ? C(0) : yv[c];
          if (MODE == ST_APPLY_DOT) part += ucur[c] * out;
        }
        if (MODE != ST_RESIDUAL || yp) yp[c] = AT::out(out);
      }
      if (formp) {
        T* pp = a.pout + voff + 3 * (size_t)n;
        pp[0] = AT::out(ucur[0]);
        pp[1] = AT::out(ucur[1]);
        pp[2] = AT::out(ucur[2]);
      }
    }
    if (MODE == ST_APPLY_DOT) {
      ucur[0] = u_l1[0];
      ucur[1] = u_l1[1];
      ucur[2] = u_l1[2];
    }
  }
  pdl_release();
  if (MODE != ST_APPLY) {
    C pv[1] = {out_xy ? part : C(0)};
    double o[1];
    block_sum_to_f64<1>(pv, red, o);
    const int nparts = gridDim.x * gridDim.y;
    double* parts = a.partials + (size_t)rhs * nparts;
    if (threadIdx.x == 0) parts[blockIdx.y * gridDim.x + blockIdx.x] = o[0];
    if (MODE == ST_APPLY_DOT && a.st && a.counter) {
      __shared__ bool s_last;
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) s_last = atomicAdd(&a.counter[rhs], 1u) == (unsigned)nparts - 1u;
      __syncthreads();
      if (s_last) {
        __threadfence();
        const double pap = sum_partials(parts, nparts, 1, 0);
        if (threadIdx.x == 0) {
          CGState& S = a.st[rhs];
          if (!(pap > 0.0) || !isfinite(pap)) {
            S.status = isfinite(pap) ? -3 : -5;
            S.done = 1;
            const_cast<int*>(a.done)[rhs] = 1;
          } else {
            S.alpha = S.rz / pap;
          }
          a.counter[rhs] = 0u;
        }
      }
    }
  }
}

}  // namespace afd

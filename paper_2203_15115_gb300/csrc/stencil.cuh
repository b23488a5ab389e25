// Matrix-free stiffness apply y = K u on the voxel hex8 mesh (Sec. 3.5: the
// system is solved without assembling K; the cost is memory traffic).
//
// Design (sm_103a): a CTA owns a TX x TY column of elements in (x, y) and marches
// through a range of z node planes.  Per element layer it stages the next node
// plane of u (3 components, masked at fixed DOFs) in shared memory, every
// thread applies E_e * K0 to one element in the Walsh-Hadamard modal form
// (afd_common.cuh), writes the 24 element forces to shared memory (SoA, bank
// conflict free), and each node thread gathers the 4 bottom-face forces of the
// layer above and the 4 top-face forces of the layer below.  Neighbouring CTAs
// overlap by one element column so that every node is finished by exactly one
// CTA: no atomics, deterministic sums.
#pragma once

#include "afd_common.cuh"

namespace afd {

enum StencilMode {
  ST_APPLY = 0,     // y = K u
  ST_RESIDUAL = 1,  // y = f - K u, partial sum y.y, optional float copy of y
  ST_APPLY_DOT = 2  // y = K u, partial sum u.y
};

template <typename T, typename TF>
struct StencilArgs {
  Grid gr;
  const T* u;             // [rhs][ndof]
  T* y;                   // [rhs][ndof]
  const T* E;             // [nelem] element moduli in the working type
  const uint8_t* fixed;   // [nnodes] bit c set = DOF c fixed (nullable: none fixed)
  ElemConsts<T> K;
  const TF* f;            // ST_RESIDUAL: [rhs][ndof]
  float* y32;             // ST_RESIDUAL: optional float copy of y
  double* partials;       // [rhs][nblocks] (ST_RESIDUAL, ST_APPLY_DOT)
  const int* done;        // [rhs] skip the work when nonzero (nullable)
  int kz;                 // node planes per CTA
  int tiles_x;            // CTAs along x
};

template <typename T, int TX, int TY, int MODE, typename TF>
__global__ void __launch_bounds__(TX * TY)
stencil_kernel(const StencilArgs<T, TF> a) {
  constexpr int NT = TX * TY;
  constexpr int PX = TX + 1, PY = TY + 1;     // node plane tile
  __shared__ T us[2][3][PY][PX];
  __shared__ T eo[24][TY][TX];
  __shared__ double red[32 * 1];

  const int rhs = blockIdx.z;
  if (a.done && a.done[rhs]) return;
  const Grid gr = a.gr;
  const int tile_x = blockIdx.x % a.tiles_x;
  const int tile_y = blockIdx.x / a.tiles_x;
  const int ex0 = tile_x * (TX - 1) - 1;
  const int ey0 = tile_y * (TY - 1) - 1;
  const int k0 = blockIdx.y * a.kz;
  const int k1 = min(k0 + a.kz, gr.nnz);
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const size_t voff = (size_t)rhs * gr.ndof;
  const T* __restrict__ u = a.u + voff;
  T* __restrict__ y = a.y + voff;

  auto load_plane = [&](int kn, int slot) {
    // nodes [ex0, ex0+TX] x [ey0, ey0+TY] of plane kn, AoS rows of 3*PX values
    for (int q = threadIdx.x; q < 3 * PX * PY; q += NT) {
      const int row = q / (3 * PX);
      const int w = q - row * 3 * PX;
      const int nxl = w / 3;
      const int c = w - nxl * 3;
      const int i = ex0 + nxl, j = ey0 + row;
      T val = T(0);
      if (kn >= 0 && kn < gr.nnz && i >= 0 && i < gr.nnx && j >= 0 && j < gr.nny) {
        const int n = i + gr.nnx * (j + gr.nny * kn);
        const bool fx = a.fixed ? ((a.fixed[n] >> c) & 1) : false;
        val = fx ? T(0) : u[3 * (size_t)n + c];
      }
      us[slot][c][row][nxl] = val;
    }
  };

  // node owned by this thread (interior of the element tile)
  const int ni = ex0 + tx, nj = ey0 + ty;
  const bool node_thread = tx >= 1 && ty >= 1 && ni <= gr.nx && nj <= gr.ny;
  T acc[3] = {T(0), T(0), T(0)};
  T part = T(0);
  const int ei = ex0 + tx, ej = ey0 + ty;
  const bool elem_xy = ei >= 0 && ei < gr.nx && ej >= 0 && ej < gr.ny;

  load_plane(k0 - 1, (k0 - 1) & 1);
  for (int l = k0 - 1; l < k1; ++l) {
    load_plane(l + 1, (l + 1) & 1);
    __syncthreads();
    // ---- element (ei, ej, l) ----
    {
      T E = T(0);
      if (elem_xy && l >= 0 && l < gr.nz) E = a.E[ei + gr.nx * (ej + gr.ny * l)];
      T v[3][8];
      if (E != T(0)) {
#pragma unroll
        for (int az = 0; az < 2; ++az) {
          const int s = (l + az) & 1;
#pragma unroll
          for (int ay = 0; ay < 2; ++ay)
#pragma unroll
            for (int ax = 0; ax < 2; ++ax)
#pragma unroll
              for (int c = 0; c < 3; ++c) v[c][ax + 2 * ay + 4 * az] = us[s][c][ty + ay][tx + ax];
        }
        hex8_apply(v, E, a.K);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int q = 0; q < 8; ++q) v[c][q] = T(0);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) eo[3 * q + c][ty][tx] = v[c][q];
    }
    __syncthreads();
    // ---- nodes of plane l (bottom faces of layer l + top faces of layer l-1) ----
    if (node_thread) {
      T top[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const int la = (1 - dx) + 2 * (1 - dy);  // our local index in element (tx-1+dx, ty-1+dy)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            acc[c] += eo[3 * la + c][ty - 1 + dy][tx - 1 + dx];
            top[c] += eo[3 * (la + 4) + c][ty - 1 + dy][tx - 1 + dx];
          }
        }
      if (l >= k0) {
        const int n = ni + gr.nnx * (nj + gr.nny * l);
        const uint8_t fb = a.fixed ? a.fixed[n] : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const bool fx = (fb >> c) & 1;
          T out;
          if (MODE == ST_RESIDUAL) {
            out = fx ? T(0) : (T)a.f[voff + 3 * (size_t)n + c] - acc[c];
            part += out * out;
            if (a.y32) a.y32[voff + 3 * (size_t)n + c] = (float)out;
          } else {
            out = fx ? T(0) : acc[c];
            if (MODE == ST_APPLY_DOT) part += us[l & 1][c][ty][tx] * out;
          }
          y[3 * (size_t)n + c] = out;
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] = top[c];
    }
    __syncthreads();
  }
  if (MODE != ST_APPLY) {
    T pv[1] = {part};
    double out[1];
    block_sum_to_f64<1>(pv, red, out);
    if (threadIdx.x == 0) a.partials[(size_t)rhs * gridDim.x * gridDim.y + blockIdx.y * gridDim.x + blockIdx.x] = out[0];
  }
}

// Launch geometry of the stencil for a grid.
template <int TX, int TY>
struct StencilGeom {
  static void get(const Grid& gr, int kz, int& tiles_x, dim3& grid) {
    tiles_x = (gr.nnx + (TX - 2)) / (TX - 1);
    const int tiles_y = (gr.nny + (TY - 2)) / (TY - 1);
    const int zch = (gr.nnz + kz - 1) / kz;
    grid = dim3(tiles_x * tiles_y, zch, 1);
  }
};

}  // namespace afd

// Common device code of the assembly-free deflated FE path (arXiv 2203.15115,
// Sec. 3.5): grid geometry, the hex8 element operator in Walsh-Hadamard modal
// form, and deterministic block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include "dfloat.cuh"

namespace afd {

// ----------------------------------------------------------------------------
// Grid geometry.  Node (i,j,k): n = i + nnx*(j + nny*k); element e = i + nx*(j + ny*k).
// ----------------------------------------------------------------------------
struct Grid {
  int nx, ny, nz;     // elements per axis
  int nnx, nny, nnz;  // nodes per axis (= n? + 1)
  int nnodes;         // nnx*nny*nnz
  int nelem;          // nx*ny*nz
  int ndof;           // 3*nnodes
  int vs;             // per-RHS stride of the device vectors: ndof rounded up to a multiple of 4
};

// Deflation groups: node (i,j,k) -> (min(i/g, ngx-1), ...).
struct Groups {
  int g;
  int ngx, ngy, ngz, ng;
  double h;  // element edge, for the node coordinates x = h*i
};

__host__ __device__ inline int group_of_axis(int i, int g, int ng) {
  int G = i / g;
  return G < ng ? G : ng - 1;
}

// Centroid of the nodes of group G along one axis: the node planes of the
// group are [g*G, g*G+g-1], the last group also takes the planes up to n_nodes-1.
__host__ __device__ inline double group_centroid_axis(int G, int g, int ng, int nn, double h) {
  int lo = g * G;
  int hi = (G == ng - 1) ? (nn - 1) : (g * G + g - 1);
  return 0.5 * h * (double)(lo + hi);
}

// ----------------------------------------------------------------------------
// Element operator constants.  The element stiffness of the trilinear cube of
// edge h with unit modulus is applied as y = H^T grad_h W(H u): H is the 8-point
// Walsh-Hadamard transform of each displacement component (sums/differences
// over the element's nodes) and W the element strain energy written in the
// orthogonal modal basis {1, x, y, z, xy, yz, zx, xyz} of the cube.  Per
// element this is ~180 flops instead of the 1152 of a dense 24x24 product.
//
// With lam, mu the Lame parameters of E = 1 and the modal coefficients h_m of
// the Walsh-Hadamard transform, the energy is
//   W = Phi(A)/16 + [Phi(Hx) + Phi(Hy) + Phi(Hz)]/48 + [sum of xyz terms]/144
// (Phi(F) = lam/2 tr(F)^2 + mu |sym F|^2; A the 9 linear coefficients, Hx/Hy/Hz
// the bilinear coefficients arranged as gradient tensors), all scaled by h.
// ----------------------------------------------------------------------------
template <typename T>
struct ElemConsts {
  T l16;     // lam/16
  T m16;     // mu/16
  T m8;      // 2 mu/16
  T l48;     // lam/48
  T m48;     // mu/48
  T m3_48;   // 3 mu/48
  T t144;    // (lam + 4 mu)/144
};

template <typename T>
__host__ inline ElemConsts<T> make_elem_consts(double nu, double h) {
  double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double mu = 1.0 / (2.0 * (1.0 + nu));
  ElemConsts<T> c;
  c.l16 = (T)(h * lam / 16.0);
  c.m16 = (T)(h * mu / 16.0);
  c.m8 = (T)(h * 2.0 * mu / 16.0);
  c.l48 = (T)(h * lam / 48.0);
  c.m48 = (T)(h * mu / 48.0);
  c.m3_48 = (T)(h * 3.0 * mu / 48.0);
  c.t144 = (T)(h * (lam + 4.0 * mu) / 144.0);
  return c;
}

// Diagonal of the unit-modulus element matrix: (lam + 4 mu)/9 * h (every entry).
__host__ inline double elem_diag(double nu, double h) {
  double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double mu = 1.0 / (2.0 * (1.0 + nu));
  return h * (lam + 4.0 * mu) / 9.0;
}

// Forward transform of 8 nodal values (local node a = ax + 2ay + 4az):
// out[m] = sum_a prod_{bits b of m} (2 a_b - 1) * v[a].
template <typename T>
__device__ __forceinline__ void wht8_fwd(T (&v)[8]) {
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int bit = 1 << b;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      if (!(a & bit)) {
        T x0 = v[a], x1 = v[a | bit];
        v[a] = x0 + x1;
        v[a | bit] = x1 - x0;
      }
    }
  }
}

// Transposed transform: out[a] = sum_m prod_{bits b of m} (2 a_b - 1) * g[m].
template <typename T>
__device__ __forceinline__ void wht8_tr(T (&g)[8]) {
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int bit = 1 << b;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      if (!(a & bit)) {
        T x0 = g[a], x1 = g[a | bit];
        g[a] = x0 - x1;
        g[a | bit] = x0 + x1;
      }
    }
  }
}

// Modal forces: given the transformed displacement h[c][m] (in place), replace
// it by d W / d h scaled by the element modulus E (h[c][0] becomes 0).
template <typename T>
__device__ __forceinline__ void modal_forces(T (&h)[3][8], T E, const ElemConsts<T>& K) {
  const T l16 = K.l16 * E, m16 = K.m16 * E, m8 = K.m8 * E;
  const T l48 = K.l48 * E, m48 = K.m48 * E, m3 = K.m3_48 * E, t144 = K.t144 * E;
  // linear block: A_dj = h[d][1<<j]
  {
    const T Axx = h[0][1], Ayy = h[1][2], Azz = h[2][4];
    const T tr = l16 * (Axx + Ayy + Azz);
    const T sxy = m16 * (h[0][2] + h[1][1]);
    const T syz = m16 * (h[1][4] + h[2][2]);
    const T szx = m16 * (h[2][1] + h[0][4]);
    h[0][1] = fma(m8, Axx, tr);
    h[1][2] = fma(m8, Ayy, tr);
    h[2][4] = fma(m8, Azz, tr);
    h[0][2] = sxy; h[1][1] = sxy;
    h[1][4] = syz; h[2][2] = syz;
    h[2][1] = szx; h[0][4] = szx;
  }
  // bilinear block: P = h[.][3] (xy), Q = h[.][6] (yz), R = h[.][5] (zx)
  {
    const T Px = h[0][3], Py = h[1][3], Pz = h[2][3];
    const T Qx = h[0][6], Qy = h[1][6], Qz = h[2][6];
    const T Rx = h[0][5], Ry = h[1][5], Rz = h[2][5];
    const T s1 = l48 * (Px + Qz);
    const T s2 = l48 * (Py + Rz);
    const T s3 = l48 * (Rx + Qy);
    const T s = Pz + Qx + Ry;
    h[0][3] = fma(m3, Px, s1);
    h[2][6] = fma(m3, Qz, s1);
    h[1][3] = fma(m3, Py, s2);
    h[2][5] = fma(m3, Rz, s2);
    h[0][5] = fma(m3, Rx, s3);
    h[1][6] = fma(m3, Qy, s3);
    h[2][3] = m48 * (Pz + s);
    h[0][6] = m48 * (Qx + s);
    h[1][5] = m48 * (Ry + s);
  }
  // trilinear block (diagonal)
  h[0][7] *= t144;
  h[1][7] *= t144;
  h[2][7] *= t144;
  h[0][0] = T(0);
  h[1][0] = T(0);
  h[2][0] = T(0);
}

// y_e = E * K0 * u_e for one element; u[c][a] -> overwritten with y[c][a].
template <typename T>
__device__ __forceinline__ void hex8_apply(T (&u)[3][8], T E, const ElemConsts<T>& K) {
  wht8_fwd(u[0]);
  wht8_fwd(u[1]);
  wht8_fwd(u[2]);
  modal_forces(u, E, K);
  wht8_tr(u[0]);
  wht8_tr(u[1]);
  wht8_tr(u[2]);
}

// ----------------------------------------------------------------------------
// Programmatic dependent launch (sm_90+): a kernel launched with the
// programmatic-serialization attribute may start while its predecessor in the
// stream is finishing.  pdl_release() lets the successor start launching once
// every CTA of this grid has begun; pdl_acquire() waits until the predecessor
// grid has completed and its writes are visible.  Both are no-ops for a
// normal launch.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_acquire() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ----------------------------------------------------------------------------
// Reductions.  Values are summed per thread in the working type, combined
// across the warp in the working type, and across warps and blocks in FP64 in
// a fixed order (deterministic).
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of NV values per thread into FP64; result valid in thread 0.
// `scratch` must hold 32*NV doubles.  blockDim.x must be a multiple of 32.
// Warp trees in the working type, then thread q adds value q over the warps
// in order (deterministic).
template <int NV, typename T>
__device__ __forceinline__ void block_sum_to_f64(T (&v)[NV], double* scratch, double (&out)[NV]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    T w = warp_sum(v[q]);
    if (lane == 0) scratch[q * 32 + warp] = (double)w;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nwarps; ++w) s += scratch[threadIdx.x * 32 + w];
    scratch[threadIdx.x * 32] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) out[q] = scratch[q * 32];
  }
  __syncthreads();
}

}  // namespace afd

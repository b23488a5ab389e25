// FP32 matrix-free stiffness apply y = K u, two node rows per thread with the
// two element rows packed into the lanes of one float2 (Sec. 3.5: K is never
// assembled; the cost of an iteration is the operator apply).
//
// Design (sm_103a).  The modal hex8 operator and the column march are those
// of stencil.cuh: every thread owns node columns and marches along z, the x
// butterflies go through warp shuffles, the y butterflies through shared
// memory, the z butterflies stay in registers.  Here a thread owns the two
// node rows jb = base + 2w and jb + 1 of its column and computes the two
// element rows A (between jb and jb+1) and B (between jb+1 and jb+2) at once:
// every value of the element pipeline is a float2 (A in .x, B in .y), so each
// butterfly, each modal-force product and each transposed butterfly is one
// packed FP32 instruction (FADD2/FFMA2/FMUL2 of sm_100+) for two elements.
// Only row jb+2 comes from the next warp (shared memory), so a CTA of TY
// warps covers 2 TY node rows and finishes 2 TY - 2 of them, with one barrier
// per exchange for two nodes per thread.  The arithmetic of each element is
// the same sequence of correctly rounded operations as in stencil.cuh.
#pragma once

#include "afd_common.cuh"
#include "dpcg_kernels.cuh"
#include "stencil.cuh"
#include "packed.cuh"

namespace afd {

// Launch geometry: a CTA of TY warps covers 2 TY node rows, finishes rows
// base+1 .. base+2TY-2 (2 TY - 2 of them), and (ST_TX - 2) columns over kz planes.
template <int TY>
struct StencilGeom2 {
  static constexpr int ROWS = 2 * TY - 2;
  static void get(const Grid& gr, int kz, int& tiles_x, dim3& grid) {
    tiles_x = (gr.nnx + (ST_TX - 3)) / (ST_TX - 2);
    const int tiles_y = (gr.nny + ROWS - 1) / ROWS;
    const int zch = (gr.nnz + kz - 1) / kz;
    grid = dim3(tiles_x * tiles_y, zch, 1);
  }
};

// Load policies for the vectors the stencil reads: LoadRO for data that no
// CTA of the running kernel writes (read-only cache path), LoadCG for data
// written by other CTAs of the same (persistent) kernel, read from L2.
struct LoadRO {
  template <typename X>
  __device__ __forceinline__ static X ld(const X* p) { return __ldg(p); }
};
struct LoadCG {
  template <typename X>
  __device__ __forceinline__ static X ld(const X* p) { return __ldcg(p); }
};
// Weak load cached in L1 (ld.global.ca): for data written by other CTAs
// before a grid-wide barrier whose acquire fence orders it (never the
// non-coherent path).
struct LoadCA {
  template <typename X>
  __device__ __forceinline__ static X ld(const X* p) { return __ldca(p); }
};

// One CTA tile (tile = tile_x + tiles_x * tile_y, z chunk zc) of one RHS.
// Returns this thread's partial sum (ST_RESIDUAL: y.y, ST_APPLY_DOT: p.Ap,
// else 0) over the nodes it finishes.  beta: ST_APPLY_DOT's search-direction
// coefficient.  Called by every thread of the CTA.
// Dynamic shared memory of the asynchronous staging ring (bytes): RING
// planes x (node values of both rows [+ z] + two fixed-mask words + two moduli)
// per thread.
constexpr int ST_RING = 3;
template <int TY, int MODE>
constexpr int stencil2_ring_floats() {
  return ST_RING * ((MODE == ST_APPLY_DOT ? 12 : 6) + 4) * ST_TX * TY;
}

template <int TY, int MODE, typename LD, bool ASYNC = false>
__device__ __forceinline__ float stencil2_tile(const StencilArgs<float, float>& a, float beta, int tile, int zc,
                                               int rhs, float* ring = nullptr) {
  // Exchange buffers (each written, then read after a barrier; the other
  // exchange's barrier separates that read from the next write):
  //   xe: (S, D) x-edge values of row jb for the warp below, per component
  //   ye: (mx = 0, 1) forces of element B on row jb + 2, for the warp above
  __shared__ float2 xe[3][TY][ST_TX];
  __shared__ float2 ye[3][TY][ST_TX];

  const Grid gr = a.gr;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tile_x = tile % a.tiles_x;
  const int tile_y = tile / a.tiles_x;
  const int i = tile_x * (ST_TX - 2) - 1 + lane;
  const int jb = tile_y * StencilGeom2<TY>::ROWS - 1 + 2 * w;   // row a = 0; row a = 1 is jb + 1
  const int k0 = zc * a.kz;
  const int k1 = min(k0 + a.kz, gr.nnz);
  const size_t voff = (size_t)rhs * gr.vs;
  const float* u = a.u + voff;

  const bool ci = i >= 0 && i < gr.nnx;
  const bool col0 = ci && jb >= 0 && jb < gr.nny;
  const bool col1 = ci && jb + 1 >= 0 && jb + 1 < gr.nny;
  const bool ei = lane < ST_TX - 1 && i >= 0 && i < gr.nx;
  const bool elA = ei && jb >= 0 && jb < gr.ny;
  const bool elB = ei && w < TY - 1 && jb + 1 >= 0 && jb + 1 < gr.ny;
  const bool oi = lane >= 1 && lane < ST_TX - 1 && i <= gr.nx;
  const bool out0 = oi && w >= 1 && jb <= gr.ny;
  const bool out1 = oi && w <= TY - 2 && jb + 1 <= gr.ny;

  // Fused search direction p = z + W mu + beta p_old (as in stencil.cuh; in
  // ST_APPLY_DOT, which the solver always launches with z).  For this column
  // the rigid motion of group G is W mu = A_G + r_z B_G per row (the two rows
  // may lie in different groups along y), A = t + omega x (r_x, r_y, 0),
  // B = (omega_y, -omega_x, 0).  A and B change only when the plane index
  // enters the next group along z; they are kept in this thread's slot of
  // shared memory (not registers) together with nothing else: the lever arms
  // are recomputed at each refresh.
  constexpr bool formp = MODE == ST_APPLY_DOT;
  const Groups gp = a.gp;
  const float hh = (float)(0.5 * gp.h);
  __shared__ float2 sAB[formp ? 5 : 1][formp ? ST_TX * TY : 1];
  int gz_next = 0;   // first plane of the next group along z (0: not loaded yet)
  int zsum = 0;      // zlo + zhi of the current group along z
  const double* murhs = formp ? a.mu + (size_t)rhs * 6 * gp.ng : nullptr;
  auto refresh_group = [&](int k) {
    const int gz = group_of_axis(k, gp.g, gp.ngz);
    int zlo, zhi, lo, hi;
    group_range(gz, gp.g, gp.ngz, gr.nz, zlo, zhi);
    gz_next = (gz == gp.ngz - 1) ? (1 << 30) : zhi + 1;
    zsum = zlo + zhi;
    if (!ci) return;
    const int Gx = group_of_axis(i, gp.g, gp.ngx);
    group_range(Gx, gp.g, gp.ngx, gr.nx, lo, hi);
    const float rx = hh * (float)(2 * i - lo - hi);
    const int j0 = max(jb, 0), j1 = min(jb + 1, gr.nny - 1);
    const int Gy0 = group_of_axis(j0, gp.g, gp.ngy), Gy1 = group_of_axis(j1, gp.g, gp.ngy);
    group_range(Gy0, gp.g, gp.ngy, gr.ny, lo, hi);
    const float ry0 = hh * (float)(2 * j0 - lo - hi);
    group_range(Gy1, gp.g, gp.ngy, gr.ny, lo, hi);
    const float ry1 = hh * (float)(2 * j1 - lo - hi);
    const int gzo = gp.ngx * gp.ngy * gz;
    const double* m0 = murhs + 6 * (Gx + gp.ngx * Gy0 + gzo);
    const double* m1 = murhs + 6 * (Gx + gp.ngx * Gy1 + gzo);
    const float tx0 = (float)LD::ld(m0), ty0 = (float)LD::ld(m0 + 1), tz0 = (float)LD::ld(m0 + 2);
    const float ox0 = (float)LD::ld(m0 + 3), oy0 = (float)LD::ld(m0 + 4), oz0 = (float)LD::ld(m0 + 5);
    const float tx1 = (float)LD::ld(m1), ty1 = (float)LD::ld(m1 + 1), tz1 = (float)LD::ld(m1 + 2);
    const float ox1 = (float)LD::ld(m1 + 3), oy1 = (float)LD::ld(m1 + 4), oz1 = (float)LD::ld(m1 + 5);
    const int me = threadIdx.x;
    sAB[0][me] = make_float2(tx0 - oz0 * ry0, tx1 - oz1 * ry1);
    sAB[1][me] = make_float2(ty0 + oz0 * rx, ty1 + oz1 * rx);
    sAB[2][me] = make_float2(tz0 + (ox0 * ry0 - oy0 * rx), tz1 + (ox1 * ry1 - oy1 * rx));
    sAB[3][me] = make_float2(oy0, oy1);
    sAB[4][me] = make_float2(-ox0, -ox1);
  };

  // (u or the formed p) of both rows at plane k; fixed bits of both rows in fbits
  auto load_node = [&](int k, float2 (&v)[3], unsigned& fbits) {
    v[0] = v[1] = v[2] = bc2(0.f);
    fbits = 0u;
    if (k < 0 || k >= gr.nnz) return;
    const int n0 = i + gr.nnx * (jb + gr.nny * k);
    const int n1 = n0 + gr.nnx;
    const unsigned f0 = (col0 && a.fixed) ? __ldg(a.fixed + n0) : 0u;
    const unsigned f1 = (col1 && a.fixed) ? __ldg(a.fixed + n1) : 0u;
    fbits = f0 | (f1 << 8);
    float p0[3] = {0.f, 0.f, 0.f}, p1[3] = {0.f, 0.f, 0.f};
    if (col0) {
      const float* q = u + 3 * (size_t)n0;
      p0[0] = LD::ld(q); p0[1] = LD::ld(q + 1); p0[2] = LD::ld(q + 2);
    }
    if (col1) {
      const float* q = u + 3 * (size_t)n1;
      p1[0] = LD::ld(q); p1[1] = LD::ld(q + 1); p1[2] = LD::ld(q + 2);
    }
    if constexpr (formp) {
      if (k >= gz_next) refresh_group(k);
      float z0[3] = {0.f, 0.f, 0.f}, z1[3] = {0.f, 0.f, 0.f};
      if (col0) {
        const float* q = a.z + voff + 3 * (size_t)n0;
        z0[0] = LD::ld(q); z0[1] = LD::ld(q + 1); z0[2] = LD::ld(q + 2);
      }
      if (col1) {
        const float* q = a.z + voff + 3 * (size_t)n1;
        z1[0] = LD::ld(q); z1[1] = LD::ld(q + 1); z1[2] = LD::ld(q + 2);
      }
      const float2 rz = bc2(hh * (float)(2 * k - zsum)), bt = bc2(beta);
      const int me = threadIdx.x;
      v[0] = fma2(bt, make_float2(p0[0], p1[0]), add2(make_float2(z0[0], z1[0]), fma2(rz, sAB[3][me], sAB[0][me])));
      v[1] = fma2(bt, make_float2(p0[1], p1[1]), add2(make_float2(z0[1], z1[1]), fma2(rz, sAB[4][me], sAB[1][me])));
      v[2] = fma2(bt, make_float2(p0[2], p1[2]), add2(make_float2(z0[2], z1[2]), sAB[2][me]));
    } else {
      v[0] = make_float2(p0[0], p1[0]);
      v[1] = make_float2(p0[1], p1[1]);
      v[2] = make_float2(p0[2], p1[2]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (!col0 || ((f0 >> c) & 1u)) v[c].x = 0.f;
      if (!col1 || ((f1 >> c) & 1u)) v[c].y = 0.f;
    }
  };

  // Asynchronous staging (ASYNC): plane k's node values (and z), the fixed-mask
  // words of its two nodes and the moduli of element layer k-1 are copied
  // into this thread's slot of a ring of ST_RING planes; consume() waits for
  // nothing itself (the caller's cp_async_wait does) and forms the values.
  constexpr int NQ = formp ? 12 : 6;
  constexpr int NT = ST_TX * TY;
  const int me = threadIdx.x;
  auto issue = [&](int k, int slot) {
    if (k <= k1) {
      const bool kin = k >= 0 && k < gr.nnz;
      const bool v0 = kin && col0, v1 = kin && col1;
      const size_t n0 = v0 ? (size_t)(i + gr.nnx * (jb + gr.nny * k)) : 0;
      const size_t n1 = v1 ? (size_t)(i + gr.nnx * (jb + 1 + gr.nny * k)) : 0;
      float* rs = ring + (size_t)slot * NQ * NT;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cp_async4(rs + c * NT + me, u + 3 * n0 + c, v0);
        cp_async4(rs + (3 + c) * NT + me, u + 3 * n1 + c, v1);
      }
      if constexpr (formp) {
        const float* zb = a.z + voff;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cp_async4(rs + (6 + c) * NT + me, zb + 3 * n0 + c, v0);
          cp_async4(rs + (9 + c) * NT + me, zb + 3 * n1 + c, v1);
        }
      }
      unsigned* fr = (unsigned*)(ring + (size_t)ST_RING * NQ * NT) + (size_t)slot * 2 * NT;
      const bool hf = a.fixed != nullptr;
      const void* fsrc0 = hf ? (const void*)(a.fixed + (n0 & ~(size_t)3)) : (const void*)u;
      const void* fsrc1 = hf ? (const void*)(a.fixed + (n1 & ~(size_t)3)) : (const void*)u;
      cp_async4(fr + me, fsrc0, v0 && hf);
      cp_async4(fr + NT + me, fsrc1, v1 && hf);
      float* er = ring + (size_t)ST_RING * (NQ + 2) * NT + (size_t)slot * 2 * NT;
      const int L = k - 1;
      const bool lin = L >= 0 && L < gr.nz;
      const size_t eA = (lin && elA) ? (size_t)(i + gr.nx * (jb + gr.ny * L)) : 0;
      const size_t eB = (lin && elB) ? (size_t)(i + gr.nx * (jb + 1 + gr.ny * L)) : 0;
      cp_async4(er + me, a.E + eA, lin && elA);
      cp_async4(er + NT + me, a.E + eB, lin && elB);
    }
    cp_async_commit();
  };
  auto consume = [&](int k, int slot, float2 (&v)[3], unsigned& fbits, float2& Eo) {
    const float* rs = ring + (size_t)slot * NQ * NT;
    const unsigned* fr = (const unsigned*)(ring + (size_t)ST_RING * NQ * NT) + (size_t)slot * 2 * NT;
    const float* er = ring + (size_t)ST_RING * (NQ + 2) * NT + (size_t)slot * 2 * NT;
    Eo = make_float2(er[me], er[NT + me]);
    const bool kin = k >= 0 && k < gr.nnz;
    const int n0 = i + gr.nnx * (jb + gr.nny * (kin ? k : 0));
    const unsigned f0 = (kin && col0) ? (fr[me] >> (8 * (n0 & 3))) & 0xffu : 0u;
    const unsigned f1 = (kin && col1) ? (fr[NT + me] >> (8 * ((n0 + gr.nnx) & 3))) & 0xffu : 0u;
    fbits = f0 | (f1 << 8);
    if constexpr (formp) {
      if (kin && k >= gz_next) refresh_group(k);
      const float2 rz = bc2(hh * (float)(2 * k - zsum)), bt = bc2(beta);
      v[0] = fma2(bt, make_float2(rs[me], rs[3 * NT + me]),
                  add2(make_float2(rs[6 * NT + me], rs[9 * NT + me]), fma2(rz, sAB[3][me], sAB[0][me])));
      v[1] = fma2(bt, make_float2(rs[NT + me], rs[4 * NT + me]),
                  add2(make_float2(rs[7 * NT + me], rs[10 * NT + me]), fma2(rz, sAB[4][me], sAB[1][me])));
      v[2] = fma2(bt, make_float2(rs[2 * NT + me], rs[5 * NT + me]),
                  add2(make_float2(rs[8 * NT + me], rs[11 * NT + me]), sAB[2][me]));
    } else {
      v[0] = make_float2(rs[me], rs[3 * NT + me]);
      v[1] = make_float2(rs[NT + me], rs[4 * NT + me]);
      v[2] = make_float2(rs[2 * NT + me], rs[5 * NT + me]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (!kin || !col0 || ((f0 >> c) & 1u)) v[c].x = 0.f;
      if (!kin || !col1 || ((f1 >> c) & 1u)) v[c].y = 0.f;
    }
  };

  // Face values of elements A and B on one node plane: F[c][q], q = mx + 2 my.
  auto face_values = [&](const float2 (&un)[3], float2 (&F)[3][4]) {
    float2 S[3], D[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 right = make_float2(__shfl_down_sync(0xffffffffu, un[c].x, 1),
                                       __shfl_down_sync(0xffffffffu, un[c].y, 1));  // lane 31: unused
      S[c] = add2(right, un[c]);
      D[c] = sub2(right, un[c]);
      xe[c][w][lane] = make_float2(S[c].x, D[c].x);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 up = (w < TY - 1) ? xe[c][w + 1][lane] : bc2(0.f);   // (S, D) of row jb + 2
      const float2 St = make_float2(S[c].y, up.x), Dt = make_float2(D[c].y, up.y);
      F[c][0] = add2(St, S[c]);
      F[c][1] = add2(Dt, D[c]);
      F[c][2] = sub2(St, S[c]);
      F[c][3] = sub2(Dt, D[c]);
    }
  };

  float2 Fb[3][4], Tprev[3][4];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) Fb[c][q] = Tprev[c][q] = bc2(0.f);

  float2 ucur[3] = {bc2(0.f), bc2(0.f), bc2(0.f)};   // formed u at plane l (dot and p write)
  unsigned fcur = 0u, fnext;
  float part = 0.f;
  float2 un[3];
  float2 Enext = bc2(0.f);   // ASYNC: moduli of the element layer below plane `un`
  if constexpr (ASYNC) {
    // plane k -> ring slot (k - k0 + 1) % ST_RING
    issue(k0 - 1, 0);
    issue(k0, 1);
    issue(k0 + 1, 2);
    cp_async_wait<2>();
    {
      float2 un0[3], Ed;
      unsigned fdummy;
      consume(k0 - 1, 0, un0, fdummy, Ed);
      face_values(un0, Fb);
      __syncthreads();  // the loop's first x-edge write follows this read
    }
    cp_async_wait<1>();
    consume(k0, 1, un, fnext, Enext);
  } else {
    {
      float2 un0[3];
      unsigned fdummy;
      load_node(k0 - 1, un0, fdummy);
      face_values(un0, Fb);
      __syncthreads();  // the loop's first x-edge write follows this read
    }
    load_node(k0, un, fnext);
  }

  for (int l = k0 - 1; l < k1; ++l) {
    float2 Ft[3][4];
    face_values(un, Ft);
    const float2 u_l1[3] = {un[0], un[1], un[2]};
    const unsigned f_l1 = fnext;
    float2 E = bc2(0.f);
    if constexpr (ASYNC) {
      E = Enext;
      issue(l + 3, (l + 3 - k0 + 1) % ST_RING);   // into the slot of plane l
    } else {
      if (l >= 0 && l < gr.nz) {
        const int e0 = i + gr.nx * (jb + gr.ny * l);
        if (elA) E.x = __ldg(a.E + e0);
        if (elB) E.y = __ldg(a.E + e0 + gr.nx);
      }
      if (l + 2 <= k1) load_node(l + 2, un, fnext);
    }

    float2 h[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int q = 1; q < 4; ++q) h[c][q] = add2(Ft[c][q], Fb[c][q]);
#pragma unroll
      for (int q = 0; q < 4; ++q) h[c][q + 4] = sub2(Ft[c][q], Fb[c][q]);
    }
    modal_forces2(h, E, a.K);
    float2 Bf[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // q = 0: the rigid-translation force is zero
      Bf[c][0] = sub2(Tprev[c][0], h[c][4]);
      Tprev[c][0] = h[c][4];
#pragma unroll
      for (int q = 1; q < 4; ++q) {
        Bf[c][q] = add2(sub2(h[c][q], h[c][q + 4]), Tprev[c][q]);
        Tprev[c][q] = add2(h[c][q], h[c][q + 4]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) Fb[c][q] = Ft[c][q];
    }

    // transposed y stage: e0 -> (row jb from A, row jb+1 from B), e1 -> (row jb+1 from A, row jb+2 from B)
    float2 e0[3][2], e1[3][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int mx = 0; mx < 2; ++mx) {
        e0[c][mx] = sub2(Bf[c][mx], Bf[c][mx + 2]);
        e1[c][mx] = add2(Bf[c][mx], Bf[c][mx + 2]);
      }
      ye[c][w][lane] = make_float2(e1[c][0].y, e1[c][1].y);
    }
    __syncthreads();
    float2 yv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 below = (w >= 1) ? ye[c][w - 1][lane] : bc2(0.f);   // element row jb-1 on row jb
      const float2 t0 = add2(e0[c][0], make_float2(below.x, e1[c][0].x));
      const float2 t1 = add2(e0[c][1], make_float2(below.y, e1[c][1].x));
      // transposed x stage: edge (i, i+1) -> node i gets s - d, node i+1 gets s + d
      const float2 sp = add2(t0, t1);
      const float2 fl = make_float2(__shfl_up_sync(0xffffffffu, sp.x, 1), __shfl_up_sync(0xffffffffu, sp.y, 1));
      yv[c] = add2(sub2(t0, t1), lane >= 1 ? fl : bc2(0.f));
    }

    if (l >= k0) {
      const int n0 = i + gr.nnx * (jb + gr.nny * l);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const bool ok = r == 0 ? out0 : out1;
        if (!ok) continue;
        const int n = n0 + r * gr.nnx;
        const unsigned fb = (fcur >> (8 * r)) & 0xffu;
        float* yp = a.y + voff + 3 * (size_t)n;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float yc = r == 0 ? yv[c].x : yv[c].y;
          const float uc = r == 0 ? ucur[c].x : ucur[c].y;
          const bool fx = (fb >> c) & 1u;
          float out;
          if (MODE == ST_RESIDUAL) {
            out = fx ? 0.f : __ldg(a.f + voff + 3 * (size_t)n + c) - yc;
            part += out * out;
            if (a.y32) a.y32[voff + 3 * (size_t)n + c] = out;
          } else {
            out = fx ? 0.f : yc;
            if (MODE == ST_APPLY_DOT || MODE == ST_DOT_PLAIN) part += uc * out;
          }
          yp[c] = out;
        }
        if constexpr (formp) {
          float* pp = a.pout + voff + 3 * (size_t)n;
          pp[0] = r == 0 ? ucur[0].x : ucur[0].y;
          pp[1] = r == 0 ? ucur[1].x : ucur[1].y;
          pp[2] = r == 0 ? ucur[2].x : ucur[2].y;
        }
      }
    }
    if constexpr (ASYNC) {
      if (l + 2 <= k1) {
        cp_async_wait<1>();   // plane l+2 has landed (plane l+3 may still be in flight)
        consume(l + 2, (l + 2 - k0 + 1) % ST_RING, un, fnext, Enext);
      }
    }
    ucur[0] = u_l1[0];
    ucur[1] = u_l1[1];
    ucur[2] = u_l1[2];
    fcur = f_l1;
  }
  if constexpr (ASYNC) cp_async_wait<0>();   // no copy may land after the tile
  return MODE == ST_APPLY ? 0.f : part;
}

template <int TY, int MODE, bool ASYNC>
__global__ void __launch_bounds__(ST_TX * TY, 16 / TY)
stencil2_kernel(const StencilArgs<float, float> a) {
  __shared__ double red[32];
  pdl_acquire();
  const int rhs = blockIdx.z;
  if (a.done && a.done[rhs]) return;
  // ST_APPLY_DOT in the solver loop: beta and the stopping test from the
  // previous iteration's partials.  beta goes through shared memory so that
  // the tile can re-read it instead of holding a register across the march.
  __shared__ float s_beta;
  if (MODE == ST_APPLY_DOT) {
    if (a.ip.upd) {
      double b;
      if (!dpcg_iteration_start(a.st, rhs, const_cast<int*>(a.done), a.ip, b)) return;
      if (threadIdx.x == 0) s_beta = (float)b;
    } else {
      if (threadIdx.x == 0) s_beta = (float)a.st[rhs].beta;
    }
    __syncthreads();
  }
  const float beta = MODE == ST_APPLY_DOT ? s_beta : 0.f;
  extern __shared__ float st2_ring[];
  const float part = stencil2_tile<TY, MODE, LoadRO, ASYNC>(a, beta, blockIdx.x, blockIdx.y, rhs, st2_ring);
  pdl_release();
  if (MODE != ST_APPLY) {
    float pv[1] = {part};
    double o[1];
    block_sum_to_f64<1>(pv, red, o);
    const int nparts = gridDim.x * gridDim.y;
    double* parts = a.partials + (size_t)rhs * nparts;
    if (threadIdx.x == 0) parts[blockIdx.y * gridDim.x + blockIdx.x] = o[0];
    if ((MODE == ST_APPLY_DOT || MODE == ST_DOT_PLAIN) && a.st && a.counter) {
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

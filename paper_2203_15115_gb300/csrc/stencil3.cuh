// FP32 matrix-free stiffness apply y = K u (Sec. 3.5: K is never assembled;
// the cost of an iteration is the operator apply), with the search direction
// p = z + W mu + beta p_old of the deflated PCG iteration formed on load.
//
// Design (sm_103a).  The operator is the modal hex8 form of afd_common.cuh
// with its butterflies factorised across the grid: x stage by warp shuffle,
// y stage by one shared-memory exchange per plane, z stage in registers along
// a march over node planes.  What this kernel changes against stencil2.cuh is
// the bookkeeping around that arithmetic:
//  * a CTA of TY warps covers two bands of TY node rows, and every value of
//    the element pipeline is a float2 holding the same position in both bands
//    (.x band 0, .y band 1).  The bands are independent, so every butterfly,
//    force product and exchange is one packed instruction with no register
//    shuffling between the lanes of a pair, and the y exchanges move float4s
//    (both bands' pair of values) per thread;
//  * node values, element moduli (and the fixed-DOF words) are staged a few
//    planes ahead by 4-byte cp.async into a per-thread ring in shared memory,
//    addressed by 32-bit node offsets (one multiply-add per band and plane);
//  * the modal blocks (bilinear, trilinear, linear) are formed and reduced one
//    after the other, and the applied vector of the plane being finished waits
//    in shared memory, so the march fits in 128 registers (two CTAs of 8
//    warps per SM) without spilling;
//  * fixed DOFs are applied only in CTAs whose tile contains a fixed node
//    (a per-tile flag); elsewhere only the column-validity factor remains.
// Band b, warp w holds node row j = tile_y ROWS - 1 + b TY + w; lane l holds
// node column i = tile_x 30 - 1 + l.  Lanes 1..30 and every row except the
// first of band 0 and the last of band 1 are finished here (2 TY - 2 rows),
// and every node is finished by exactly one thread: no atomics, deterministic.
#pragma once

#include "afd_common.cuh"
#include "dpcg_kernels.cuh"
#include "packed.cuh"
#include "stencil.cuh"

namespace afd {

constexpr int ST3_RING = 3;   // planes per thread in the staging ring (2 in flight while one is used)
constexpr int ST3_COLS = ST_TX - 2;

// RP = false: two row bands per CTA (2 TY - 2 finished rows); RP = true: one
// band of TY rows and two load cases in the lanes of every float2 (TY - 2
// finished rows).
template <int TY, bool RP = false>
struct St3Geom {
  static constexpr int ROWS = RP ? TY - 2 : 2 * TY - 2;
  static void get(const Grid& gr, int kz, int& tiles_x, int& tiles_y, dim3& grid) {
    tiles_x = (gr.nnx + ST3_COLS - 1) / ST3_COLS;
    tiles_y = (gr.nny + ROWS - 1) / ROWS;
    grid = dim3(tiles_x * tiles_y, (gr.nnz + kz - 1) / kz, 1);
  }
};

// Ring values per thread and plane: u (3 per band or load case), z (3 per
// band or load case, formed search direction only), the modulus of the
// element layer below the plane (per band; the pair mode uses the first), the
// 4-byte word holding the node's fixed bits (likewise).
template <int MODE>
struct St3Q {
  static constexpr bool FORMP = MODE == ST_APPLY_DOT;
  static constexpr int U = 0;
  static constexpr int Z = 6;
  static constexpr int E = FORMP ? 12 : 6;
  static constexpr int F = E + 2;
  static constexpr int N = F + 2;
};

template <int TY, int MODE>
constexpr size_t st3_smem_bytes() {
  // ring + x-edge exchange (TY + 1 warp slots) + y exchange (TY + 1 slots), float4 per component,
  // + the rigid-motion coefficients A, B of the search direction (5 float2 per thread)
  return (size_t)ST3_RING * St3Q<MODE>::N * ST_TX * TY * 4 + 2 * (size_t)3 * (TY + 1) * ST_TX * 16 +
         (St3Q<MODE>::FORMP ? (size_t)5 * ST_TX * TY * 8 : 0) + (size_t)6 * ST_TX * TY * 8;   // + sP
}

// Tiles whose loaded window (30 x ROWS output nodes plus a one-node halo on
// each side in x and y) holds a node with a fixed DOF, over all planes.  One
// CTA per tile.
template <int TY, bool RP>
__global__ void k_st3_tile_flags(const Grid gr, const uint8_t* __restrict__ fixed, int tiles_x, uint8_t* flags) {
  constexpr int ROWS = St3Geom<TY, RP>::ROWS;
  const int tile = blockIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int i0 = max(tx * ST3_COLS - 1, 0), i1 = min(tx * ST3_COLS + ST3_COLS + 1, gr.nnx);
  const int j0 = max(ty * ROWS - 1, 0), j1 = min(ty * ROWS + ROWS + 1, gr.nny);
  const int ni = i1 - i0, nj = j1 - j0;
  int any = 0;
  if (fixed && ni > 0 && nj > 0) {
    const long long cnt = (long long)ni * nj * gr.nnz;
    for (long long t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int di = (int)(t % ni);
      const long long r = t / ni;
      const int dj = (int)(r % nj);
      const int k = (int)(r / nj);
      if (fixed[(size_t)(i0 + di) + (size_t)gr.nnx * ((size_t)(j0 + dj) + (size_t)gr.nny * k)]) any = 1;
    }
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) flags[tile] = (uint8_t)any;
}

// One CTA tile (tile_x, tile_y, z chunk zc) of one RHS (RP: of the load
// cases rhs0 in the .x lanes and rhs1 in the .y lanes, each only where act0 /
// act1); returns this thread's partial sums (.x band 0 or rhs0, .y band 1 or
// rhs1) over the nodes it finishes: p.(K p) (ST_APPLY_DOT / ST_DOT_PLAIN) or
// r.r with r = f - K u written in place of y (ST_RESIDUAL).
template <int TY, int MODE, bool MASKED, bool RP>
__device__ __forceinline__ float2 st3_tile(const StencilArgs<float, float>& a, float2 beta, int tile, int zc, int rhs0,
                                           int rhs1, bool act0, bool act1, float* smem) {
  using Q = St3Q<MODE>;
  constexpr bool formp = Q::FORMP;
  constexpr bool dot = MODE == ST_APPLY_DOT || MODE == ST_DOT_PLAIN;
  constexpr int NT = ST_TX * TY;
  const Grid gr = a.gr;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int tile_x = tile % a.tiles_x, tile_y = tile / a.tiles_x;
  const int i = tile_x * ST3_COLS - 1 + lane;
  // rows of band 0 and band 1 (one row for both load cases in the pair mode)
  const int j0 = tile_y * St3Geom<TY, RP>::ROWS - 1 + w, j1 = RP ? j0 : j0 + TY;
  const int k0 = zc * a.kz, k1 = min(k0 + a.kz, gr.nnz);
  const size_t voff0 = (size_t)rhs0 * gr.vs, voff1 = (size_t)(RP ? rhs1 : rhs0) * gr.vs;
  const int PS = gr.nnx * gr.nny, ES = gr.nx * gr.ny;

  float* ring = smem;
  float4* xe = reinterpret_cast<float4*>(smem + ST3_RING * Q::N * NT);   // [3][TY + 1][32]
  float4* ye = xe + 3 * (TY + 1) * ST_TX;                                  // [3][TY + 1][32]
  float2* sAB = reinterpret_cast<float2*>(ye + 3 * (TY + 1) * ST_TX);      // [5][NT] (formed p only)
  float2* sP = sAB + (formp ? 5 * NT : 0);                                 // [2][3][NT] applied vector by plane parity

  // column validity (nodes and elements) per band, fixed for the tile
  const bool ci = i >= 0 && i < gr.nnx;
  const bool cv0 = ci && j0 >= 0 && j0 < gr.nny, cv1 = ci && j1 >= 0 && j1 < gr.nny;
  const bool ei = i >= 0 && i < gr.nx;
  const bool ev0 = ei && j0 >= 0 && j0 < gr.ny, ev1 = ei && j1 >= 0 && j1 < gr.ny;
  const bool oi = lane >= 1 && lane <= ST3_COLS && i < gr.nnx;
  const bool ov0 = RP ? act0 && oi && w >= 1 && w <= TY - 2 && cv0 : oi && w >= 1 && cv0;
  const bool ov1 = RP ? act1 && oi && w >= 1 && w <= TY - 2 && cv1 : oi && w <= TY - 2 && cv1;
  // node offsets of plane 0 (the element below-left of node (i, j) has offset n - j)
  const int n0 = cv0 ? i + gr.nnx * j0 : 0, n1 = cv1 ? i + gr.nnx * j1 : 0;

  const float* u0 = a.u + voff0;
  const float* u1 = a.u + voff1;
  const float* zv0 = formp ? a.z + voff0 : nullptr;
  const float* zv1 = formp ? a.z + voff1 : nullptr;
  // producer state: the next plane to stage and its ring slot
  int pk = k0 - 1, pslot = 0;
  auto issue = [&]() {
    float* rs = ring + pslot * (Q::N * NT) + tid;
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(rs);
    const bool kin = pk >= 0 && pk < gr.nnz;
    const bool lin = pk >= 1 && pk <= gr.nz;
    const int pn0 = kin && cv0 ? n0 + pk * PS : 0, pn1 = kin && cv1 ? n1 + pk * PS : 0;
    const int pe0 = lin && ev0 ? n0 - j0 + (pk - 1) * ES : 0, pe1 = lin && ev1 ? n1 - j1 + (pk - 1) * ES : 0;
    const int sz0 = kin && cv0 ? 4 : 0, sz1 = kin && cv1 ? 4 : 0;
    const float* a0 = u0 + 3 * (size_t)pn0;
    const float* a1 = u1 + 3 * (size_t)pn1;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sbase + (Q::U + c) * NT * 4),
                   "l"(a0 + c), "r"(sz0) : "memory");
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sbase + (Q::U + 3 + c) * NT * 4),
                   "l"(a1 + c), "r"(sz1) : "memory");
    }
    if constexpr (formp) {
      const float* b0 = zv0 + 3 * (size_t)pn0;
      const float* b1 = zv1 + 3 * (size_t)pn1;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sbase + (Q::Z + c) * NT * 4),
                     "l"(b0 + c), "r"(sz0) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sbase + (Q::Z + 3 + c) * NT * 4),
                     "l"(b1 + c), "r"(sz1) : "memory");
      }
    }
    {
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sbase + Q::E * NT * 4), "l"(a.E + pe0),
                   "r"(lin && ev0 ? 4 : 0) : "memory");
      if constexpr (!RP)   // the pair's load cases share the element row
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sbase + (Q::E + 1) * NT * 4),
                     "l"(a.E + pe1), "r"(lin && ev1 ? 4 : 0) : "memory");
    }
    if constexpr (MASKED) {
      const uint8_t* f0 = a.fixed + ((size_t)pn0 & ~(size_t)3);
      const uint8_t* f1 = a.fixed + ((size_t)pn1 & ~(size_t)3);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sbase + Q::F * NT * 4), "l"(f0),
                   "r"(sz0) : "memory");
      if constexpr (!RP)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sbase + (Q::F + 1) * NT * 4), "l"(f1),
                     "r"(sz1) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    ++pk;
    pslot = pslot + 1 == ST3_RING ? 0 : pslot + 1;
  };

  // Rigid motion W mu of the groups of this column (search direction only):
  // per band A + r_z B with A = t + omega x (r_x, r_y, 0), B = (omega_y, -omega_x)
  // (z component of B is 0), refreshed when the plane enters a new group along z.
  const Groups gp = a.gp;
  const float hh = (float)(0.5 * gp.h);
  int gz_next = -(1 << 30), zsum = 0;
  const double* murhs0 = formp ? a.mu + (size_t)rhs0 * 6 * gp.ng : nullptr;
  const double* murhs1 = formp ? a.mu + (size_t)(RP ? rhs1 : rhs0) * 6 * gp.ng : nullptr;
  auto refresh_group = [&](int k) {
    const int gz = group_of_axis(k, gp.g, gp.ngz);
    int zlo, zhi, lo, hi;
    group_range(gz, gp.g, gp.ngz, gr.nz, zlo, zhi);
    gz_next = (gz == gp.ngz - 1) ? (1 << 30) : zhi + 1;
    zsum = zlo + zhi;
    const int ic = min(max(i, 0), gr.nnx - 1);
    const int Gx = group_of_axis(ic, gp.g, gp.ngx);
    group_range(Gx, gp.g, gp.ngx, gr.nx, lo, hi);
    const float rx = hh * (float)(2 * ic - lo - hi);
    const int jc0 = min(max(j0, 0), gr.nny - 1), jc1 = min(max(j1, 0), gr.nny - 1);
    const int Gy0 = group_of_axis(jc0, gp.g, gp.ngy), Gy1 = group_of_axis(jc1, gp.g, gp.ngy);
    group_range(Gy0, gp.g, gp.ngy, gr.ny, lo, hi);
    const float ry0 = hh * (float)(2 * jc0 - lo - hi);
    group_range(Gy1, gp.g, gp.ngy, gr.ny, lo, hi);
    const float ry1 = hh * (float)(2 * jc1 - lo - hi);
    const int gzo = gp.ngx * gp.ngy * gz;
    const double* m0 = murhs0 + 6 * (Gx + gp.ngx * Gy0 + gzo);
    const double* m1 = murhs1 + 6 * (Gx + gp.ngx * Gy1 + gzo);
    const float tx0 = (float)__ldg(m0), ty0 = (float)__ldg(m0 + 1), tz0 = (float)__ldg(m0 + 2);
    const float ox0 = (float)__ldg(m0 + 3), oy0 = (float)__ldg(m0 + 4), oz0 = (float)__ldg(m0 + 5);
    const float tx1 = (float)__ldg(m1), ty1 = (float)__ldg(m1 + 1), tz1 = (float)__ldg(m1 + 2);
    const float ox1 = (float)__ldg(m1 + 3), oy1 = (float)__ldg(m1 + 4), oz1 = (float)__ldg(m1 + 5);
    sAB[0 * NT + tid] = make_float2(tx0 - oz0 * ry0, tx1 - oz1 * ry1);
    sAB[1 * NT + tid] = make_float2(ty0 + oz0 * rx, ty1 + oz1 * rx);
    sAB[2 * NT + tid] = make_float2(tz0 + (ox0 * ry0 - oy0 * rx), tz1 + (ox1 * ry1 - oy1 * rx));
    sAB[3 * NT + tid] = make_float2(oy0, oy1);
    sAB[4 * NT + tid] = make_float2(-ox0, -ox1);
  };

  // consumer state
  int cslot = 0;
  const float2 bt = beta;
  // The values of plane k from the ring: the applied vector v (u, or the
  // formed p), with its fixed DOFs (MASKED) and invalid columns zeroed; the
  // fixed bits of both bands (bits 0-2 band 0, 8-10 band 1, MASKED only) and
  // E of the element layer below the plane.
  auto consume = [&](int k, float2 (&v)[3], unsigned& fb, float2& E) {
    const float* rs = ring + cslot * (Q::N * NT) + tid;
    cslot = cslot + 1 == ST3_RING ? 0 : cslot + 1;
    E = RP ? bc2(rs[Q::E * NT]) : make_float2(rs[Q::E * NT], rs[(Q::E + 1) * NT]);
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = make_float2(rs[(Q::U + c) * NT], rs[(Q::U + 3 + c) * NT]);
    if constexpr (formp) {
      if (k >= 0 && k < gr.nnz) {   // uniform; outside the mesh the staged zeros stand
        if (k >= gz_next) refresh_group(k);
        const float2 rz = bc2(hh * (float)(2 * k - zsum));
        const float2 cz = make_float2(cv0 ? 1.f : 0.f, cv1 ? 1.f : 0.f);
        float2 zz[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) zz[c] = make_float2(rs[(Q::Z + c) * NT], rs[(Q::Z + 3 + c) * NT]);
        v[0] = mul2(cz, fma2(bt, v[0], add2(zz[0], fma2(rz, sAB[3 * NT + tid], sAB[0 * NT + tid]))));
        v[1] = mul2(cz, fma2(bt, v[1], add2(zz[1], fma2(rz, sAB[4 * NT + tid], sAB[1 * NT + tid]))));
        v[2] = mul2(cz, fma2(bt, v[2], add2(zz[2], sAB[2 * NT + tid])));
      }
    }
    if constexpr (MASKED) {
      const unsigned w0 = __float_as_uint(rs[Q::F * NT]), w1 = RP ? w0 : __float_as_uint(rs[(Q::F + 1) * NT]);
      fb = ((w0 >> (8 * ((n0 + k * PS) & 3))) & 7u) | (((w1 >> (8 * ((n1 + k * PS) & 3))) & 7u) << 8);
#pragma unroll
      for (int c = 0; c < 3; ++c)
        v[c] = mul2(v[c], make_float2(((fb >> c) & 1u) ? 0.f : 1.f, ((fb >> (8 + c)) & 1u) ? 0.f : 1.f));
    }
  };

  // x-edges (S, D) of the plane held in v, both bands: exchanged through
  // shared memory with the warp below (which needs the row above it); warp 0
  // also fills the slot above the last warp with its band-1 values as band 0
  // (the last warp's band-0 row is followed by band 1's first row).
  auto faces = [&](const float2 (&v)[3], float2 (&F)[3][4]) {
    float2 S[3], D[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 right = make_float2(__shfl_down_sync(0xffffffffu, v[c].x, 1), __shfl_down_sync(0xffffffffu, v[c].y, 1));
      S[c] = add2(right, v[c]);
      D[c] = sub2(right, v[c]);
      xe[(c * (TY + 1) + w) * ST_TX + lane] = make_float4(S[c].x, S[c].y, D[c].x, D[c].y);
    }
    if (!RP && w == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) xe[(c * (TY + 1) + TY) * ST_TX + lane] = make_float4(S[c].y, 0.f, D[c].y, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 up = xe[(c * (TY + 1) + w + 1) * ST_TX + lane];
      const float2 Su = make_float2(up.x, up.y), Du = make_float2(up.z, up.w);
      F[c][0] = add2(Su, S[c]);
      F[c][1] = add2(Du, D[c]);
      F[c][2] = sub2(Su, S[c]);
      F[c][3] = sub2(Du, D[c]);
    }
  };

  const ElemConsts<float>& K = a.K;
  float2 FA[3][4], FB[3][4], Tprev[3][4];
  float2 PA[3];
  unsigned MA = 0u, MB = 0u;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) Tprev[c][q] = bc2(0.f);
  float2 part = bc2(0.f);

  // prologue: three planes in flight, plane k0 - 1 made into the bottom faces
  if constexpr (RP) {
    // the slot above the last warp (x-edges) and below the first (y forces)
    // belong to no warp in the pair mode: zeros, for rows that are not finished
    if (w == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        xe[(c * (TY + 1) + TY) * ST_TX + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        ye[(c * (TY + 1)) * ST_TX + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  if constexpr (formp) {
#pragma unroll
    for (int q = 0; q < 5; ++q) sAB[q * NT + tid] = bc2(0.f);
  }
  issue();
  issue();
  issue();
  cp_async_wait<2>();
  {
    float2 E;
    consume(k0 - 1, PA, MA, E);
    if constexpr (dot) {
#pragma unroll
      for (int c = 0; c < 3; ++c) sP[(((k0 - 1) & 1) * 3 + c) * NT + tid] = PA[c];
    }
  }
  faces(PA, FA);
  __syncthreads();   // every read of the prologue's exchange precedes the march's first write

  // One step: element layer l between node planes l and l + 1.  In: Fb (faces
  // of plane l), Mc (fixed bits of plane l; its applied vector waits in sP).
  // Out: Ft (faces of plane l + 1), Mn, the applied vector of plane l + 1 (Pn,
  // and in sP); y (and p) of plane l when l >= k0.  The
  // modal blocks are formed and reduced one at a time (bilinear, trilinear,
  // linear) so that the transformed values of the three never live at once;
  // each value still sees the same operations in the same order.
  auto step = [&](int l, float2 (&Fb)[3][4], float2 (&Ft)[3][4], float2 (&Pn)[3], unsigned Mc, unsigned& Mn) {
    issue();
    cp_async_wait<2>();
    float2 E;
    consume(l + 1, Pn, Mn, E);
    if constexpr (dot) {
#pragma unroll
      for (int c = 0; c < 3; ++c) sP[(((l + 1) & 1) * 3 + c) * NT + tid] = Pn[c];
    }
    faces(Pn, Ft);
    float2 Bf[3][4];
    {
      // bilinear block: P = h[.][3] (xy), Q = h[.][6] (yz), R = h[.][5] (zx)
      float2 P[3], Qv[3], R[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        P[c] = add2(Ft[c][3], Fb[c][3]);
        R[c] = sub2(Ft[c][1], Fb[c][1]);
        Qv[c] = sub2(Ft[c][2], Fb[c][2]);
      }
      const float2 l48 = mul2(bc2(K.l48), E), m48 = mul2(bc2(K.m48), E), m3 = mul2(bc2(K.m3_48), E);
      {
        const float2 s1 = mul2(l48, add2(P[0], Qv[2]));
        const float2 s2 = mul2(l48, add2(P[1], R[2]));
        const float2 s3 = mul2(l48, add2(R[0], Qv[1]));
        const float2 sm = add2(add2(P[2], Qv[0]), R[1]);
        const float2 fP0 = fma2(m3, P[0], s1), fQ2 = fma2(m3, Qv[2], s1);
        const float2 fP1 = fma2(m3, P[1], s2), fR2 = fma2(m3, R[2], s2);
        const float2 fR0 = fma2(m3, R[0], s3), fQ1 = fma2(m3, Qv[1], s3);
        const float2 fP2 = mul2(m48, add2(P[2], sm));
        const float2 fQ0 = mul2(m48, add2(Qv[0], sm));
        const float2 fR1 = mul2(m48, add2(R[1], sm));
        P[0] = fP0; P[1] = fP1; P[2] = fP2;
        Qv[0] = fQ0; Qv[1] = fQ1; Qv[2] = fQ2;
        R[0] = fR0; R[1] = fR1; R[2] = fR2;
      }
      // trilinear block h[.][7] and the z pair (3, 7)
      const float2 t144 = mul2(bc2(K.t144), E);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 f7 = mul2(sub2(Ft[c][3], Fb[c][3]), t144);
        Bf[c][3] = add2(sub2(P[c], f7), Tprev[c][3]);
        Tprev[c][3] = add2(P[c], f7);
      }
      // linear block: A_dj = h[d][1 << j], h[.][4] = Ft[.][0] - Fb[.][0]
      float2 L1[3], L2[3], L4[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        L1[c] = add2(Ft[c][1], Fb[c][1]);
        L2[c] = add2(Ft[c][2], Fb[c][2]);
        L4[c] = sub2(Ft[c][0], Fb[c][0]);
      }
      const float2 l16 = mul2(bc2(K.l16), E), m16 = mul2(bc2(K.m16), E), m8 = mul2(bc2(K.m8), E);
      {
        const float2 Axx = L1[0], Ayy = L2[1], Azz = L4[2];
        const float2 tr = mul2(l16, add2(add2(Axx, Ayy), Azz));
        const float2 sxy = mul2(m16, add2(L2[0], L1[1]));
        const float2 syz = mul2(m16, add2(L4[1], L2[2]));
        const float2 szx = mul2(m16, add2(L1[2], L4[0]));
        L1[0] = fma2(m8, Axx, tr);
        L2[1] = fma2(m8, Ayy, tr);
        L4[2] = fma2(m8, Azz, tr);
        L2[0] = sxy; L1[1] = sxy;
        L4[1] = syz; L2[2] = syz;
        L1[2] = szx; L4[0] = szx;
      }
      // z pairs (1, 5), (2, 6), (0, 4); the rigid-translation force is zero
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Bf[c][1] = add2(sub2(L1[c], R[c]), Tprev[c][1]);
        Tprev[c][1] = add2(L1[c], R[c]);
        Bf[c][2] = add2(sub2(L2[c], Qv[c]), Tprev[c][2]);
        Tprev[c][2] = add2(L2[c], Qv[c]);
        Bf[c][0] = sub2(Tprev[c][0], L4[c]);
        Tprev[c][0] = L4[c];
      }
    }
    // transposed y stage: e0 -> this node row, e1 -> the row above (through
    // the exchange to the warp above; the last warp's band 0 goes to warp 0's band 1)
    float2 e0[3][2], e1[3][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int mx = 0; mx < 2; ++mx) {
        e0[c][mx] = sub2(Bf[c][mx], Bf[c][mx + 2]);
        e1[c][mx] = add2(Bf[c][mx], Bf[c][mx + 2]);
      }
      ye[(c * (TY + 1) + w + 1) * ST_TX + lane] = make_float4(e1[c][0].x, e1[c][0].y, e1[c][1].x, e1[c][1].y);
    }
    if (!RP && w == TY - 1) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
        ye[(c * (TY + 1)) * ST_TX + lane] = make_float4(0.f, e1[c][0].x, 0.f, e1[c][1].x);
    }
    __syncthreads();
    float2 yv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 bl = ye[(c * (TY + 1) + w) * ST_TX + lane];
      const float2 t0 = add2(e0[c][0], make_float2(bl.x, bl.y));
      const float2 t1 = add2(e0[c][1], make_float2(bl.z, bl.w));
      // transposed x stage: edge (i-1, i) gives node i its s + d
      const float2 sp = add2(t0, t1);
      const float2 fl = make_float2(__shfl_up_sync(0xffffffffu, sp.x, 1), __shfl_up_sync(0xffffffffu, sp.y, 1));
      yv[c] = add2(sub2(t0, t1), fl);
    }
    if (l >= k0) {
      if constexpr (MASKED && MODE != ST_RESIDUAL) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          yv[c] = mul2(yv[c], make_float2(((Mc >> c) & 1u) ? 0.f : 1.f, ((Mc >> (8 + c)) & 1u) ? 0.f : 1.f));
      }
      float2 Pl[3];
      if constexpr (dot) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Pl[c] = sP[((l & 1) * 3 + c) * NT + tid];
          part = fma2(mul2(Pl[c], make_float2(ov0 ? 1.f : 0.f, ov1 ? 1.f : 0.f)), yv[c], part);
        }
      }
      const size_t o0 = voff0 + 3 * (size_t)(n0 + l * PS), o1 = voff1 + 3 * (size_t)(n1 + l * PS);
      if constexpr (MODE == ST_RESIDUAL) {
        // r = f - K u on the free DOFs (0 on fixed DOFs), its partial r.r, optional float copy
        const float* f = a.f;
        const float2 ov2 = make_float2(ov0 ? 1.f : 0.f, ov1 ? 1.f : 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float2 r = sub2(make_float2(ov0 ? __ldg(f + o0 + c) : 0.f, ov1 ? __ldg(f + o1 + c) : 0.f), yv[c]);
          if constexpr (MASKED)
            r = mul2(r, make_float2(((Mc >> c) & 1u) ? 0.f : 1.f, ((Mc >> (8 + c)) & 1u) ? 0.f : 1.f));
          yv[c] = r;
          r = mul2(r, ov2);
          part = fma2(r, r, part);
        }
        if (a.y32) {
          if (ov0) {
            a.y32[o0] = yv[0].x;
            a.y32[o0 + 1] = yv[1].x;
            a.y32[o0 + 2] = yv[2].x;
          }
          if (ov1) {
            a.y32[o1] = yv[0].y;
            a.y32[o1 + 1] = yv[1].y;
            a.y32[o1 + 2] = yv[2].y;
          }
        }
      }
      float* y = a.y;
      if (ov0) {
        y[o0] = yv[0].x;
        y[o0 + 1] = yv[1].x;
        y[o0 + 2] = yv[2].x;
      }
      if (ov1) {
        y[o1] = yv[0].y;
        y[o1 + 1] = yv[1].y;
        y[o1 + 2] = yv[2].y;
      }
      if constexpr (formp) {
        float* p = a.pout;
        if (ov0) {
          p[o0] = Pl[0].x;
          p[o0 + 1] = Pl[1].x;
          p[o0 + 2] = Pl[2].x;
        }
        if (ov1) {
          p[o1] = Pl[0].y;
          p[o1 + 1] = Pl[1].y;
          p[o1 + 2] = Pl[2].y;
        }
      }
    }
  };

  for (int l = k0 - 1; l < k1; ++l) {
    step(l, FA, FB, PA, MA, MB);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int q = 0; q < 4; ++q) FA[c][q] = FB[c][q]; }
    MA = MB;
  }
  cp_async_wait<0>();   // no copy may land after the tile
  return part;
}

// RP = false: blockIdx.z is the RHS.  RP = true: blockIdx.z is the pair of
// load cases (2 z, 2 z + 1) of the nrhs (the last pair of an odd count has one).
template <int TY, int MODE, bool RP>
__global__ void __launch_bounds__(ST_TX * TY, 16 / TY)
st3_kernel(const StencilArgs<float, float> a, const uint8_t* __restrict__ tflags, int nrhs) {
  __shared__ double red[64];
  pdl_acquire();
  const int rhs0 = RP ? 2 * (int)blockIdx.z : (int)blockIdx.z;
  const int rhs1 = RP && rhs0 + 1 < nrhs ? rhs0 + 1 : rhs0;
  bool act0 = !(a.done && a.done[rhs0]);
  bool act1 = RP ? rhs1 != rhs0 && !(a.done && a.done[rhs1]) : act0;
  if (!act0 && !act1) return;
  __shared__ float s_beta[2];
  if (MODE == ST_APPLY_DOT) {
    if (a.ip.upd) {
      // the iteration start of each load case (every CTA sums the same partials and takes the same decision)
      double b;
      if (act0) {
        act0 = dpcg_iteration_start(a.st, rhs0, const_cast<int*>(a.done), a.ip, b);
        if (threadIdx.x == 0) s_beta[0] = (float)b;
      }
      if (RP && act1) {
        act1 = dpcg_iteration_start(a.st, rhs1, const_cast<int*>(a.done), a.ip, b);
        if (threadIdx.x == 0) s_beta[1] = (float)b;
      }
      if (!RP) act1 = act0;
      if (!act0 && !act1) return;
    } else {
      if (threadIdx.x == 0) {
        s_beta[0] = (float)a.st[rhs0].beta;
        s_beta[1] = (float)a.st[rhs1].beta;
      }
    }
    __syncthreads();
  }
  const float2 beta = MODE == ST_APPLY_DOT ? make_float2(s_beta[0], RP ? s_beta[1] : s_beta[0]) : bc2(0.f);
  extern __shared__ float4 st3_smem4[];
  float* smem = reinterpret_cast<float*>(st3_smem4);
  // tiles without a fixed node skip the fixed-DOF factors (uniform per CTA)
  const bool masked = a.fixed && (!tflags || tflags[blockIdx.x]);
  float2 part;
  if (masked)
    part = st3_tile<TY, MODE, true, RP>(a, beta, blockIdx.x, blockIdx.y, rhs0, rhs1, act0, act1, smem);
  else
    part = st3_tile<TY, MODE, false, RP>(a, beta, blockIdx.x, blockIdx.y, rhs0, rhs1, act0, act1, smem);
  pdl_release();
  if (MODE != ST_APPLY) {
    const int nparts = gridDim.x * gridDim.y;
    const int slot = blockIdx.y * gridDim.x + blockIdx.x;
    if constexpr (RP) {
      float pv[2] = {part.x, part.y};
      double o[2];
      block_sum_to_f64<2>(pv, red, o);
      if (threadIdx.x == 0) {
        if (act0) a.partials[(size_t)rhs0 * nparts + slot] = o[0];
        if (act1) a.partials[(size_t)rhs1 * nparts + slot] = o[1];
      }
      return;   // the last-CTA step length is not used with load-case pairs
    }
    float pv[1] = {part.x + part.y};
    double o[1];
    block_sum_to_f64<1>(pv, red, o);
    const int rhs = rhs0;
    double* parts = a.partials + (size_t)rhs * nparts;
    if (threadIdx.x == 0) parts[slot] = o[0];
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

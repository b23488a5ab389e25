// The FP32 inner deflated PCG iterations (Sec. 3.5) as one persistent,
// cooperatively launched kernel.
//
// One iteration is four phases separated by grid-wide barriers:
//   S  the stencil forms p = z + W mu + beta p_old while applying q = K p, and
//      leaves one p.q partial per CTA tile;
//   U  alpha = rho / p.q (every CTA sums the tile partials itself, in the
//      same order), x += alpha p, r -= alpha q, z = M^-1 r, per-CTA partials
//      of r.z and r.r;
//   C  the coarse right-hand side per (group, share): (W^T r)_G and
//      (W^T r)_G - (K W_G)^T z;
//   M  mu = E^-1 v (one warp per coarse row), per-CTA partials of
//      (W^T r).mu; after the barrier every CTA forms rho = r.z + (W^T r).mu,
//      beta = rho / rho_old and the convergence test from the same partials
//      in the same order, so all CTAs agree without another barrier.
// The vectors and partials written in one phase are read in a later phase by
// other CTAs: those reads go through L2 (LoadCG, __ldcg), never through the
// non-coherent read-only path.  The grid barrier's waits are bounded: a wait
// that runs out sets an error flag, every CTA leaves, and the host reports it.
#pragma once

#include "afd_common.cuh"
#include "dpcg_kernels.cuh"
#include "stencil2.cuh"
#include "gridsync.cuh"

namespace afd {

struct PersistArgs {
  StencilArgs<float, float> sa;   // gr, E, fixed, K, kz, tiles_x, gp; u/pout/y/z/mu set per iteration
  int ntiles;                     // stencil tiles per RHS (tiles_x * tiles_y * z chunks)
  int nrhs;
  float* x;
  float* r;
  float* z;
  float* q;
  float* P0;
  float* P1;
  const float* invd;
  // coarse space
  int nc, nsplit;
  const long long* aw_off;
  const int* aw_node;
  const float* AW;
  const float* Einv;              // nc x nc, row-major
  double* mu;                     // [rhs][nc]
  double* rec;                    // [rhs][ng][nsplit][12]
  // per-CTA partials
  double* part_st;                // [rhs][ntiles]
  double* part_up;                // [rhs][nblocks][4]: r.z, r.r, (W^T r).mu, unused
  CGState* st;                    // [rhs]
  int* done;                      // [rhs]
  GridBarrier* bar;
  unsigned long long* ptime;      // [10] CTA 0: ns per phase (S, U, C, M, scalars), iterations, barrier wait (S..M)
};

constexpr int PERSIST_MAX_RHS = 64;

// Coarse right-hand side of one (group, share) of one RHS: 12 FP64 values
// ((W^T r)_G, (W^T r)_G - (K W_G)^T z) written to rec (k_coarse_rhs without
// the last-block combination: phase M adds the shares).
__device__ __forceinline__ void coarse_rhs_item(const PersistArgs& a, int G, int sp, int rhs, double* red) {
  const Grid& gr = a.sa.gr;
  const Groups& gp = a.sa.gp;
  const int Gx = G % gp.ngx, Gy = (G / gp.ngx) % gp.ngy, Gz = G / (gp.ngx * gp.ngy);
  int ilo, ihi, jlo, jhi, klo, khi;
  group_range(Gx, gp.g, gp.ngx, gr.nx, ilo, ihi);
  group_range(Gy, gp.g, gp.ngy, gr.ny, jlo, jhi);
  group_range(Gz, gp.g, gp.ngz, gr.nz, klo, khi);
  const float hh = (float)(0.5 * gp.h);
  const size_t off = (size_t)rhs * gr.vs;
  float s[12];
#pragma unroll
  for (int t = 0; t < 12; ++t) s[t] = 0.f;
  {
    const int lz = khi - klo + 1;
    const int kper = (lz + a.nsplit - 1) / a.nsplit;
    const int kb = klo + sp * kper, ke = min(kb + kper, khi + 1);
    group_wtr_planes(gr, (const float*)a.r, off, ilo, ihi, jlo, jhi, klo, khi, kb, ke, hh, s,
                     [](const float* p) { return __ldcg(p); });
  }
  {
    const long long base = __ldg(a.aw_off + G);
    const int nG = (int)((__ldg(a.aw_off + G + 1) - base) / 18);
    const float* aw = a.AW + base;
    const int* nodes = a.aw_node + base / 18;
    const int per = (nG + a.nsplit - 1) / a.nsplit;
    const int qb = sp * per, qe = min(qb + per, nG);
#pragma unroll 2
    for (int t = qb + threadIdx.x; t < qe; t += blockDim.x) {
      const float* zp = a.z + off + 3 * (size_t)__ldg(nodes + t);
      const float z0 = __ldcg(zp), z1 = __ldcg(zp + 1), z2 = __ldcg(zp + 2);
#pragma unroll
      for (int m = 0; m < 6; ++m)
        s[6 + m] += __ldg(aw + (size_t)m * nG + t) * z0 + __ldg(aw + (size_t)(6 + m) * nG + t) * z1 +
                    __ldg(aw + (size_t)(12 + m) * nG + t) * z2;
    }
  }
  double o[12];
  block_sum_to_f64<12>(s, red, o);
  if (threadIdx.x == 0) {
    double* mine = a.rec + (((size_t)rhs * gp.ng + G) * a.nsplit + sp) * 12;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      mine[m] = o[m];
      mine[6 + m] = o[m] - o[6 + m];
    }
  }
}

// Sum of n partials (stride `stride`, component `comp`) written by other CTAs
// of this kernel, in a fixed order; the result reaches every thread.
__device__ __forceinline__ double sum_partials_cg(const double* p, int n, int stride, int comp) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += __ldcg(p + (size_t)i * stride + comp);
  return block_sum_bcast(s);
}

template <int TY>
__global__ void __launch_bounds__(ST_TX * TY, 16 / TY)
k_dpcg_persistent(const PersistArgs a) {
  extern __shared__ double vsh[];          // nc coarse values (phase M)
  __shared__ double red[32 * 12];
  __shared__ double s_rz[PERSIST_MAX_RHS], s_alpha[PERSIST_MAX_RHS], s_beta[PERSIST_MAX_RHS];
  __shared__ double s_rr[PERSIST_MAX_RHS];
  __shared__ int s_done[PERSIST_MAX_RHS], s_iters[PERSIST_MAX_RHS], s_status[PERSIST_MAX_RHS];
  __shared__ int s_any;

  const Grid& gr = a.sa.gr;
  const Groups& gp = a.sa.gp;
  const int nb = gridDim.x;
  const int nrhs = a.nrhs;
  unsigned int gen = 0;
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
    const CGState S = a.st[r];
    s_rz[r] = S.rz;
    s_beta[r] = S.beta;
    s_alpha[r] = 0.0;
    s_rr[r] = S.rr;
    s_done[r] = S.done;
    s_iters[r] = S.iters;
    s_status[r] = S.status;
  }
  __syncthreads();
  bool ok = true;
  // phase timing of CTA 0 (thread 0), kept in shared memory: [0..4] phases,
  // [5..8] barrier waits, [9] previous mark, [10] last arrival
  __shared__ unsigned long long s_t[11];
  const bool timing = a.ptime && blockIdx.x == 0 && threadIdx.x == 0;
  if (timing) {
    for (int q = 0; q < 9; ++q) s_t[q] = 0ull;
    s_t[9] = global_ns();
  }
  unsigned long long* parr = timing ? &s_t[10] : nullptr;
  auto mark = [&](int ph) {
    if (timing) {
      const unsigned long long t = global_ns();
      s_t[ph] += t - s_t[9];
      s_t[9] = t;
    }
  };
  int iters_run = 0;

  for (int it = 0;; ++it) {
    if (threadIdx.x == 0) {
      int any = 0;
      for (int r = 0; r < nrhs; ++r) any |= !s_done[r];
      s_any = any;
    }
    __syncthreads();
    if (!s_any) break;
    ++iters_run;
    float* pold = (it & 1) ? a.P1 : a.P0;
    float* pnew = (it & 1) ? a.P0 : a.P1;

    // ---- S: p = z + W mu + beta p_old, q = K p, per-tile p.q
    {
      StencilArgs<float, float> sa = a.sa;
      sa.u = pold;
      sa.pout = pnew;
      sa.y = a.q;
      sa.z = a.z;
      sa.mu = a.mu;
      const int ntxy = sa.tiles_x * ((gr.nny + StencilGeom2<TY>::ROWS - 1) / StencilGeom2<TY>::ROWS);
      for (int item = blockIdx.x; item < a.ntiles * nrhs; item += nb) {
        const int rhs = item / a.ntiles, t = item % a.ntiles;
        if (s_done[rhs]) continue;
        const int txy = t % ntxy, zc = t / ntxy;
        float pv[1] = {stencil2_tile<TY, ST_APPLY_DOT, LoadCA>(sa, (float)s_beta[rhs], txy, zc, rhs)};
        double o[1];
        block_sum_to_f64<1>(pv, red, o);
        if (threadIdx.x == 0) a.part_st[(size_t)rhs * a.ntiles + t] = o[0];
      }
    }
    if (!(ok = grid_barrier(a.bar, gen, parr))) break;
    if (timing) s_t[5 + 0] += global_ns() - s_t[10];
    mark(0);

    // ---- U: alpha, then x, r, z and the partials of r.z, r.r
    for (int rhs = 0; rhs < nrhs; ++rhs) {
      if (s_done[rhs]) continue;
      const double pap = sum_partials_cg(a.part_st + (size_t)rhs * a.ntiles, a.ntiles, 1, 0);
      if (threadIdx.x == 0) {
        if (!(pap > 0.0) || !isfinite(pap)) {
          s_status[rhs] = isfinite(pap) ? -3 : -5;
          s_done[rhs] = 1;
        } else {
          s_alpha[rhs] = s_rz[rhs] / pap;
        }
      }
      __syncthreads();
      if (s_done[rhs]) continue;
      const float alpha = (float)s_alpha[rhs];
      const size_t off = (size_t)rhs * gr.vs;
      float sacc[2] = {0.f, 0.f};
      const int nvec = gr.ndof / 4;
      float4* __restrict__ xv = (float4*)(a.x + off);
      float4* __restrict__ rv = (float4*)(a.r + off);
      float4* __restrict__ zv = (float4*)(a.z + off);
      const float4* pv = (const float4*)(pnew + off);
      const float4* qv = (const float4*)(a.q + off);
      const float4* dv = (const float4*)a.invd;
      const int stride = nb * blockDim.x;
      auto upd = [&](float4& xx, float4& rr, const float4& pp, const float4& qq, const float4& dd, float4& zz) {
        xx.x = fmaf(alpha, pp.x, xx.x); xx.y = fmaf(alpha, pp.y, xx.y);
        xx.z = fmaf(alpha, pp.z, xx.z); xx.w = fmaf(alpha, pp.w, xx.w);
        rr.x = fmaf(-alpha, qq.x, rr.x); rr.y = fmaf(-alpha, qq.y, rr.y);
        rr.z = fmaf(-alpha, qq.z, rr.z); rr.w = fmaf(-alpha, qq.w, rr.w);
        zz.x = rr.x * dd.x; zz.y = rr.y * dd.y; zz.z = rr.z * dd.z; zz.w = rr.w * dd.w;
        sacc[0] += rr.x * zz.x; sacc[0] += rr.y * zz.y; sacc[0] += rr.z * zz.z; sacc[0] += rr.w * zz.w;
        sacc[1] += rr.x * rr.x; sacc[1] += rr.y * rr.y; sacc[1] += rr.z * rr.z; sacc[1] += rr.w * rr.w;
      };
      for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nvec; t += 2 * stride) {
        const int t2 = t + stride;
        const bool two = t2 < nvec;
        float4 xa = __ldcg(xv + t), ra = __ldcg(rv + t);
        const float4 pa = __ldcg(pv + t), qa = __ldcg(qv + t), da = __ldg(dv + t);
        float4 xb, rb, pb, qb, db;
        if (two) {
          xb = __ldcg(xv + t2); rb = __ldcg(rv + t2);
          pb = __ldcg(pv + t2); qb = __ldcg(qv + t2); db = __ldg(dv + t2);
        }
        float4 za, zb;
        upd(xa, ra, pa, qa, da, za);
        xv[t] = xa;
        rv[t] = ra;
        zv[t] = za;
        if (two) {
          upd(xb, rb, pb, qb, db, zb);
          xv[t2] = xb;
          rv[t2] = rb;
          zv[t2] = zb;
        }
      }
      for (int d = nvec * 4 + blockIdx.x * blockDim.x + threadIdx.x; d < gr.ndof; d += nb * blockDim.x) {
        const size_t i = off + d;
        a.x[i] = fmaf(alpha, __ldcg(pnew + i), __ldcg(a.x + i));
        const float rn = fmaf(-alpha, __ldcg(a.q + i), __ldcg(a.r + i));
        a.r[i] = rn;
        const float zn = rn * __ldg(a.invd + d);
        a.z[i] = zn;
        sacc[0] += rn * zn;
        sacc[1] += rn * rn;
      }
      double o[2];
      block_sum_to_f64<2>(sacc, red, o);
      if (threadIdx.x == 0) {
        a.part_up[((size_t)rhs * nb + blockIdx.x) * 4 + 0] = o[0];
        a.part_up[((size_t)rhs * nb + blockIdx.x) * 4 + 1] = o[1];
      }
    }
    if (!(ok = grid_barrier(a.bar, gen, parr))) break;
    if (timing) s_t[5 + 1] += global_ns() - s_t[10];
    mark(1);

    // ---- C: coarse right-hand side per (group, share)
    {
      const int per_rhs = gp.ng * a.nsplit;
      for (int item = blockIdx.x; item < per_rhs * nrhs; item += nb) {
        const int rhs = item / per_rhs, t = item % per_rhs;
        if (s_done[rhs]) continue;
        coarse_rhs_item(a, t / a.nsplit, t % a.nsplit, rhs, red);
      }
    }
    if (!(ok = grid_barrier(a.bar, gen, parr))) break;
    if (timing) s_t[5 + 2] += global_ns() - s_t[10];
    mark(2);

    // ---- M: mu = Einv v, per-CTA partial of (W^T r).mu
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
      const int nc = a.nc;
      for (int rhs = 0; rhs < nrhs; ++rhs) {
        if (s_done[rhs]) continue;
        // rows of this CTA: row = (blockIdx.x + nb * j) * nwarps + warp
        const bool has_rows = blockIdx.x * nwarps < nc;
        double cd = 0.0;
        if (has_rows) {
          const double* rr = a.rec + (size_t)rhs * gp.ng * a.nsplit * 12;
          for (int qq = threadIdx.x; qq < nc; qq += blockDim.x) {
            const int G = qq / 6, c = qq % 6;
            double v = 0.0;
            for (int s2 = 0; s2 < a.nsplit; ++s2) v += __ldcg(rr + ((size_t)G * a.nsplit + s2) * 12 + 6 + c);
            vsh[qq] = v;
          }
          __syncthreads();
          for (int base = blockIdx.x * nwarps; base < nc; base += nb * nwarps) {
            const int row = base + warp;
            if (row < nc) {
              const float* er = a.Einv + (size_t)row * nc;
              float s = 0.f;
              for (int c = lane; c < nc; c += 32) s = fmaf(__ldg(er + c), (float)vsh[c], s);
              s = warp_sum(s);
              if (lane == 0) {
                a.mu[(size_t)rhs * nc + row] = (double)s;
                const int G = row / 6, c = row % 6;
                double wr = 0.0;
                for (int s2 = 0; s2 < a.nsplit; ++s2) wr += __ldcg(rr + ((size_t)G * a.nsplit + s2) * 12 + c);
                cd += wr * (double)s;
              }
            }
          }
          __syncthreads();   // vsh is rewritten for the next RHS
        }
        const double cdb = block_sum_bcast(cd);
        if (threadIdx.x == 0) a.part_up[((size_t)rhs * nb + blockIdx.x) * 4 + 2] = cdb;
      }
    }
    if (!(ok = grid_barrier(a.bar, gen, parr))) break;
    if (timing) s_t[5 + 3] += global_ns() - s_t[10];
    mark(3);

    // ---- scalars: rho, beta, convergence (identical in every CTA)
    for (int rhs = 0; rhs < nrhs; ++rhs) {
      if (s_done[rhs]) continue;
      double ps[3] = {0.0, 0.0, 0.0};
      {
        const double* pp = a.part_up + (size_t)rhs * nb * 4;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
          const double2 v01 = __ldcg((const double2*)(pp + (size_t)b * 4));
          ps[0] += v01.x;
          ps[1] += v01.y;
          ps[2] += __ldcg(pp + (size_t)b * 4 + 2);
        }
      }
      double o3[3];
      block_sum_to_f64<3>(ps, red, o3);
      if (threadIdx.x == 0) {
        const double rz = o3[0], rr = o3[1], cd = o3[2];
        const double rho = rz + cd;
        if (!isfinite(rr) || !isfinite(rho)) {
          s_status[rhs] = -5;
          s_done[rhs] = 1;
        } else {
          s_beta[rhs] = rho / s_rz[rhs];
          s_iters[rhs] += 1;
          s_rz[rhs] = rho;
          s_rr[rhs] = rr;
          const CGState& S = a.st[rhs];
          if (rr <= S.target2) {
            s_done[rhs] = 1;
            s_status[rhs] = 0;
          } else if (s_iters[rhs] >= S.max_iters) {
            s_done[rhs] = 1;
            s_status[rhs] = -3;
          }
        }
      }
      __syncthreads();
    }
    mark(4);
  }

  if (timing) {
    for (int q = 0; q < 5; ++q) a.ptime[q] += s_t[q];
    a.ptime[5] += (unsigned long long)iters_run;
    for (int q = 0; q < 4; ++q) a.ptime[6 + q] += s_t[5 + q];
  }
  if (blockIdx.x == 0) {
    __syncthreads();
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
      CGState& S = a.st[r];
      S.rz = s_rz[r];
      S.rr = s_rr[r];
      S.alpha = s_alpha[r];
      S.beta = s_beta[r];
      S.iters = s_iters[r];
      S.done = ok ? s_done[r] : 1;
      S.status = ok ? s_status[r] : -6;   // -6: a grid-barrier wait ran out
      a.done[r] = S.done;
    }
  }
}

}  // namespace afd

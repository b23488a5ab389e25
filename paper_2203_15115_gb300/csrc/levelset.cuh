// Level-set extraction (Eq. 3.6 at the cut that meets the target volume;
// Eq. 3.17 combination): combine normalised fields in float32 with one rounding
// per operation, keep the k largest values with ties toward the lower element
// index (radix select on order-preserving 32-bit keys, then a stable
// index-ordered count of the keys equal to the cut), and write the new moduli.
#pragma once

#include "afd_common.cuh"

namespace afd {

__device__ __forceinline__ uint32_t float_key(float f) {
  f = f + 0.0f;  // -0 -> +0
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float key_float(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

// keys[e] = sum_r w_r * (f_r[e] / m_r), in float32, r ascending.
__global__ void k_combine(int n, int nrhs, const float* __restrict__ f, const float* __restrict__ w,
                          const float* __restrict__ m, float* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    float acc = 0.0f;
    for (int r = 0; r < nrhs; ++r) {
      const float scaled = m[r] > 0.0f ? __fdiv_rn(f[(size_t)r * n + e], m[r]) : 0.0f;
      const float term = __fmul_rn(w[r], scaled);
      acc = (r == 0) ? term : __fadd_rn(acc, term);
    }
    out[e] = acc;
  }
}

struct SelectState {
  uint32_t prefix, mask;
  uint64_t kk;       // rank still to find among keys matching the prefix (1-based)
  uint64_t cnt_gt;   // keys strictly greater than the final cut
  uint32_t hist[256];
};

__global__ void __launch_bounds__(256)
k_select_hist(int64_t n, const float* __restrict__ x, SelectState* st, int shift) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t prefix = st->prefix, mask = st->mask;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = float_key(x[i]);
    if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&st->hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_select_pick(SelectState* st, int shift) {
  if (threadIdx.x != 0) return;
  uint64_t above = 0;
  int b = 255;
  for (; b >= 0; --b) {
    const uint64_t c = st->hist[b];
    if (above + c >= st->kk) break;
    above += c;
  }
  if (b < 0) b = 0;  // unreachable for 1 <= kk <= count
  st->cnt_gt += above;
  st->kk -= above;
  st->prefix |= ((uint32_t)b) << shift;
  st->mask |= 0xffu << shift;
  for (int q = 0; q < 256; ++q) st->hist[q] = 0;
}

constexpr int SEL_CHUNK = 4096;

// Count of keys equal to the cut in each chunk of SEL_CHUNK elements.
__global__ void __launch_bounds__(256)
k_count_eq(int64_t n, const float* __restrict__ x, const SelectState* st, uint32_t* __restrict__ cnt) {
  __shared__ uint32_t sh[256];
  const int64_t base = (int64_t)blockIdx.x * SEL_CHUNK;
  uint32_t c = 0;
  for (int q = threadIdx.x; q < SEL_CHUNK; q += blockDim.x) {
    const int64_t i = base + q;
    if (i < n && float_key(x[i]) == st->prefix) ++c;
  }
  sh[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt[blockIdx.x] = sh[0];
}

// Exclusive scan of the chunk counts (one thread, chunk count is small).
__global__ void k_scan_counts(int nchunks, uint32_t* cnt) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint64_t s = 0;
  for (int i = 0; i < nchunks; ++i) {
    const uint32_t c = cnt[i];
    cnt[i] = (uint32_t)s;
    s += c;
  }
}

// kept[e] = key > cut, or key == cut and its rank among equal keys (index
// order) < kk.  Also writes the moduli when E64/E32 are given.
__global__ void __launch_bounds__(256)
k_mark(int64_t n, const float* __restrict__ x, const SelectState* st, const uint32_t* __restrict__ offs,
       uint8_t* __restrict__ kept, double* E64, float* E32, double e_void) {
  __shared__ uint32_t wsum[8];
  const int64_t base = (int64_t)blockIdx.x * SEL_CHUNK;
  const uint32_t cut = st->prefix;
  const uint64_t need = st->kk;
  uint64_t run = offs[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = 0; t < SEL_CHUNK; t += blockDim.x) {
    const int64_t i = base + t + threadIdx.x;
    uint32_t k = 0;
    bool eq = false;
    if (i < n) {
      k = float_key(x[i]);
      eq = (k == cut);
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, eq);
    const uint32_t before_in_warp = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = before_in_warp;
    uint32_t tot = 0;
    for (int w = 0; w < 8; ++w) {
      if (w < warp) before += wsum[w];
      tot += wsum[w];
    }
    if (i < n) {
      const bool keep = (k > cut) || (eq && (run + before) < need);
      kept[i] = keep ? 1 : 0;
      if (E64) E64[i] = keep ? 1.0 : e_void;
      if (E32) E32[i] = keep ? 1.0f : (float)e_void;
    }
    run += tot;
    __syncthreads();
  }
}

// Casting constraint (Sec. 3.7) on the combined level-set keys, in place:
// along every line of elements parallel to `axis` (0 = x, 1 = y, 2 = z) each
// half of the part (element index along the axis >= parting, or below it)
// takes, from its far face toward the parting plane,
//   key'(c) = max(key(c), nextafter(key'(c_far_neighbour), +inf)),
// a running maximum raised by one float32 step per element, so that the kept
// set of any cut is a run of elements starting at the parting plane.  Each
// line is one dependent chain of these steps; the kernels below differ only in
// how they bring the keys to the chain.
__device__ __forceinline__ float casting_step(float key, float v) { return fmaxf(key, nextafterf(v, INFINITY)); }

// Lines along y or z (strided): one thread per line, neighbouring threads on
// neighbouring elements, keys loaded CAST_U at a time ahead of the chain.
constexpr int CAST_U = 8;
__global__ void k_casting_scan_strided(int nx, int ny, int nz, int axis, int parting, float* __restrict__ keys) {
  const int nlines = axis == 1 ? nx * nz : nx * ny;
  for (int L = blockIdx.x * blockDim.x + threadIdx.x; L < nlines; L += gridDim.x * blockDim.x) {
    size_t base, stride;
    int n;
    if (axis == 1) {
      const int i = L % nx, k = L / nx;
      base = (size_t)i + (size_t)nx * ny * k;
      stride = nx;
      n = ny;
    } else {
      base = (size_t)L;        // L = i + nx j
      stride = (size_t)nx * ny;
      n = nz;
    }
    float* line = keys + base;
    if (parting < n - 1) {     // upper half, from the far face c = n-1 down to parting
      float v = line[(size_t)(n - 1) * stride];
      for (int c0 = n - 2; c0 >= parting; c0 -= CAST_U) {
        float kv[CAST_U];
#pragma unroll
        for (int u = 0; u < CAST_U; ++u)
          if (c0 - u >= parting) kv[u] = line[(size_t)(c0 - u) * stride];
#pragma unroll
        for (int u = 0; u < CAST_U; ++u)
          if (c0 - u >= parting) {
            v = casting_step(kv[u], v);
            line[(size_t)(c0 - u) * stride] = v;
          }
      }
    }
    if (parting > 1) {         // lower half, from c = 0 up to parting - 1
      float v = line[0];
      const int top = parting < n ? parting : n;
      for (int c0 = 1; c0 < top; c0 += CAST_U) {
        float kv[CAST_U];
#pragma unroll
        for (int u = 0; u < CAST_U; ++u)
          if (c0 + u < top) kv[u] = line[(size_t)(c0 + u) * stride];
#pragma unroll
        for (int u = 0; u < CAST_U; ++u)
          if (c0 + u < top) {
            v = casting_step(kv[u], v);
            line[(size_t)(c0 + u) * stride] = v;
          }
      }
    }
  }
}

// Lines along x (contiguous): a block takes CASTX_L lines and walks them in
// chunks of CASTX_CH columns in the direction of the scan.  All threads load a
// chunk into shared memory (coalesced along x), the first warp runs the
// chains (thread l on line l; rows padded by one word so that the warp's
// reads fall in distinct banks), and all threads store the chunk back.
constexpr int CASTX_L = 32, CASTX_CH = 128, CASTX_T = 256;
__global__ void __launch_bounds__(CASTX_T) k_casting_scan_x(int nx, int nlines, int parting, float* __restrict__ keys) {
  __shared__ float t[CASTX_L][CASTX_CH + 1];
  const int line0 = blockIdx.x * CASTX_L;
  const int nl = min(CASTX_L, nlines - line0);
  const int me = threadIdx.x;
  float v = 0.f;   // the chain's running value (first warp)
  auto chunk = [&](int a, int b, bool down, bool first) {
    const int w = b - a + 1;
    for (int idx = me; idx < nl * w; idx += CASTX_T) {
      const int l = idx / w, c = idx - l * w;
      t[l][c] = keys[(size_t)(line0 + l) * nx + a + c];
    }
    __syncthreads();
    if (me < nl) {
      float* row = t[me];
      if (down) {
        int c = w - 1;
        if (first) v = row[c--];
        for (; c >= 0; --c) {
          v = casting_step(row[c], v);
          row[c] = v;
        }
      } else {
        int c = 0;
        if (first) v = row[c++];
        for (; c < w; ++c) {
          v = casting_step(row[c], v);
          row[c] = v;
        }
      }
    }
    __syncthreads();
    for (int idx = me; idx < nl * w; idx += CASTX_T) {
      const int l = idx / w, c = idx - l * w;
      keys[(size_t)(line0 + l) * nx + a + c] = t[l][c];
    }
    __syncthreads();   // the next chunk's loads overwrite t
  };
  if (parting < nx - 1) {      // upper half, from the far face down to parting
    bool first = true;
    for (int b = nx - 1; b >= parting; b -= CASTX_CH) {
      chunk(max(parting, b - CASTX_CH + 1), b, true, first);
      first = false;
    }
  }
  if (parting > 1) {           // lower half, from column 0 up to parting - 1
    const int top = parting < nx ? parting : nx;
    bool first = true;
    for (int a = 0; a < top; a += CASTX_CH) {
      chunk(a, min(top - 1, a + CASTX_CH - 1), false, first);
      first = false;
    }
  }
}

}  // namespace afd

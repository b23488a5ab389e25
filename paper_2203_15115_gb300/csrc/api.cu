// C ABI of the assembly-free deflated FE hot path (include/afd.h).
//
// Host driver: owns the device state of one mesh (moduli, supports, loads,
// solution, Krylov vectors in FP32 and FP64, the coarse factor), runs the
// deflated PCG either in FP64 or as FP32 inner solves inside FP64 iterative
// refinement, with each chunk of `check_every` DPCG iterations captured once
// into a CUDA graph and replayed, and convergence decided on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <cmath>
#include <limits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/afd.h"
#include "afd_common.cuh"
#include "coarse.cuh"
#include "dpcg_kernels.cuh"
#include "levelset.cuh"
#include "sens.cuh"
#include "stencil.cuh"
#include "stencil2.cuh"
#include "stencil3.cuh"
#include "dpcg_persistent.cuh"
#include "modal.cuh"
#include "topology.h"

using namespace afd;

static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(x)                                                                              \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) return fail(AFD_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

#define TRY(x)              \
  do {                      \
    int rc_ = (x);          \
    if (rc_ != AFD_OK) return rc_; \
  } while (0)

template <typename T>
static int dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) return AFD_OK;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(AFD_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
  }
  return AFD_OK;
}

template <typename T>
static void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// Krylov workspace of one arithmetic type.
template <typename T>
struct Work {
  int cap = 0;  // RHS capacity
  T *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *t = nullptr, *b = nullptr;
  T* r2 = nullptr;       // second residual buffer (r is double-buffered across iterations)
  T* AW = nullptr;       // K W on the node shells of the groups (see k_build_aw)
  size_t aw_cap = 0;
  T* invdiag = nullptr;  // per node
  T* invd = nullptr;     // per DOF (the flat update's Jacobi factors)
  T* E = nullptr;
  ElemConsts<T> K;
  cudaGraphExec_t graph = nullptr;
  int graph_nrhs = 0;
  int64_t graph_kernels = 0;
};

struct afd_mesh {
  Grid gr;
  Groups gp;
  afd_options opt;
  int device = 0;
  cudaStream_t user = nullptr, s = nullptr;
  int fcache_kind = -1;        // the field kind fbuf holds for the current u and E (-1: none); see enter()
  cudaEvent_t ev = nullptr;
  int kz = 8;                  // node planes per CTA of the FP64 stencil
  int kz32 = 8, ty32 = 16;     // planes per CTA and warps per CTA of the FP32 stencil
  int async32 = 0;             // FP32 stencil variant: 0 register prefetch, 1 cp.async ring (stencil2.cuh),
                               // 2 packed bands (stencil3.cuh)
  uint8_t* tflags = nullptr;   // per-tile "has a fixed node" flags of the packed-band stencil
  int tflags_ty = 0;           // 2 x CTA height + pair mode they were computed for (0: stale)
  int rp32 = 0;                // 1: the packed-band stencil takes load cases in pairs (two or more cases)
  size_t tflags_cap = 0;
  bool tuned = false;          // autotuner has chosen kz32 / ty32 for this mesh
  bool pdl_now = false;        // launches being captured use programmatic dependent launch
  // state
  double* E64 = nullptr;
  uint8_t* fixed = nullptr;   // per node bits
  int nrhs = 0, cap = 0;
  double *f64 = nullptr, *u64 = nullptr;
  std::vector<double> fnorm;
  bool has_moduli = false, has_loads = false, has_solution = false;
  // shared scratch
  double* partials = nullptr;
  size_t partials_cap = 0;
  CGState* st = nullptr;
  int* done = nullptr;
  double *v = nullptr, *mu = nullptr, *wr = nullptr;
  float* fbuf = nullptr;     // per-element float fields (R * nelem)
  float* fkeys = nullptr;    // combined level-set keys
  uint8_t* kept = nullptr;
  void* sel = nullptr;       // SelectState
  uint32_t* selcnt = nullptr;
  float* fsmall = nullptr;   // small float scratch (partials of max, weights, maxima)
  // coarse
  int nc = 0;
  int nsplit = 1;              // slabs per group in the coarse right-hand side
  size_t cpart_cap = 0;        // doubles allocated in cpart
  double* Ec = nullptr;        // W^T K W, FP64 sums
  double* Einv64 = nullptr;    // its inverse, FP64 path
  float* Einv32 = nullptr;     // its inverse, mixed path
  double *gjP = nullptr, *gjB = nullptr, *gjR = nullptr;  // Gauss-Jordan scratch
  double* gjD = nullptr;       // [n_c] 1 / sqrt of the coarse matrix's diagonal
  cudaGraphExec_t gj_graph[2] = {nullptr, nullptr};       // the inversion's panel sweeps (FP32, FP64), replayed
  double* cpart = nullptr;     // coarse right-hand side partials [rhs][G][split][12]
  unsigned int* counters = nullptr;  // last-block counters: [rhs] stencil, [MAX_RHS] coarse
  double* dmax = nullptr;
  int* dstatus = nullptr;
  int* gbox = nullptr;         // [N_g][6] bounding box of the group's fixed nodes (max < min: none)
  std::vector<int> gbox_h;     // host copy
  long long* aw_off = nullptr; // [N_g + 1] offset of group G's block in AW (last: total)
  int* aw_node = nullptr;      // [aw_total / 18] node index of every shell slot
  uint4* cut = nullptr;        // records of every group's cut elements (k_build_cut_recs); null: decoded per use
  double* cpart_c = nullptr;   // [N_g][shares][36] partial sums of the coarse diagonal blocks (k_coarse_cut)
  size_t cpart_c_cap = 0;
  unsigned int* ccount = nullptr;  // [N_g] share counters of k_coarse_cut
  long long* cut_off = nullptr;  // [N_g + 1] offset of group G's records
  size_t cut_cap = 0;
  double* grec = nullptr;      // [rhs][N_g][12] per-group records of the coarse right-hand side
  double* upart = nullptr;     // [rhs][RED_BLOCKS][2] partials of the vector update
  double* updred = nullptr;    // [rhs][coarse-step blocks][2] the same, summed in one slice per coarse-step block
  size_t updred_cap = 0;
  unsigned int* gcount = nullptr;  // [rhs][N_g] split counters
  size_t aw_total = 0;         // elements of AW
  // persistent inner solver: per-CTA partials, coarse records, grid barrier
  double* ppart = nullptr;
  size_t ppart_cap = 0;
  double* prec = nullptr;
  size_t prec_cap = 0;
  GridBarrier* gbar = nullptr;
  unsigned long long* ptime = nullptr;   // [10] phase times of the persistent solver (ns), iterations, barrier waits
  // adjoint stress sensitivity: lambda, its right-hand side, d sigma_PN / d eps per element, sigma_PN per RHS
  double *lam64 = nullptr, *gadj = nullptr, *dsig = nullptr, *pn_d = nullptr;
  float* lsbuf = nullptr;      // caller fields of afd_levelset_update_fields
  size_t lsbuf_cap = 0;
  int adj_cap = 0;
  // eigen analyses: the modes (first modal_n rows of mX), the lumped mass (or
  // free-DOF mask), Gram partials, small matrices, Ritz values
  double *mX = nullptr, *mmass = nullptr, *mparts = nullptr;
  double *mA = nullptr, *mB = nullptr, *mV = nullptr, *mlam = nullptr;
  int* minfo = nullptr;
  int modal_cap = 0, modal_n = 0;
  double modal_rho = 1.0;
  bool modal_valid = false;
  // buckling: the state stress (6 x nelem); the load factors
  double *bS6 = nullptr, *bcoef = nullptr;
  bool buckling_valid = false;
  // LOBPCG blocks [X | W | P] and their A and B images, double-buffered (3 kp rows each)
  double *lS[2] = {nullptr, nullptr}, *lBS[2] = {nullptr, nullptr}, *lAS[2] = {nullptr, nullptr};
  int lobpcg_cap = 0;
  int nsplit_aw = 1;
  bool coarse_valid = false;
  Work<float> w32;
  Work<double> w64;
  int64_t launches = 0;       // kernels launched (graph replays count their nodes)
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    int cur;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Order the mesh stream after the user's stream (device inputs made there).
// Start of every call on a mesh.  Any call may change u, the moduli or the
// load cases, so the cached field in fbuf is dropped here; afd_sensitivity
// refills it, and a level-set update of the same kind that follows it
// directly reuses it.
static int enter(afd_mesh* m) {
  m->fcache_kind = -1;
  CK(cudaEventRecord(m->ev, m->user));
  CK(cudaStreamWaitEvent(m->s, m->ev, 0));
  return AFD_OK;
}

static int finish(afd_mesh* m) {
  CK(cudaStreamSynchronize(m->s));
  CK(cudaGetLastError());
  return AFD_OK;
}

// layout of the small float scratch: [flag | per-RHS maxima | per-RHS weights | max partials]
constexpr int MAX_RHS = 64;
constexpr int FS_MAXV = 64;
constexpr int FS_WEIGHTS = FS_MAXV + MAX_RHS;
constexpr int FS_PARTS = FS_WEIGHTS + MAX_RHS;
constexpr int FS_MAX_BLOCKS = RED_BLOCKS / 2;
constexpr int FSMALL_SIZE = FS_PARTS + MAX_RHS * FS_MAX_BLOCKS;

// Kernel launch with programmatic dependent launch (pdl = true) or a plain
// stream-ordered launch; the kernels call pdl_release()/pdl_acquire().
template <typename... KArgs, typename... Args>
static cudaError_t launch_ex(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args... args) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

static int grid_blocks(size_t n, int threads = 256, int cap = RED_BLOCKS) {
  size_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (int)std::min<size_t>(b, (size_t)cap);
}

// Captured DPCG graphs bake in buffer addresses: drop them whenever a buffer moves.
static void invalidate_graphs(afd_mesh* m) {
  if (m->w32.graph) { cudaGraphExecDestroy(m->w32.graph); m->w32.graph = nullptr; }
  if (m->w64.graph) { cudaGraphExecDestroy(m->w64.graph); m->w64.graph = nullptr; }
}

static int ensure_partials(afd_mesh* m, size_t n) {
  if (n <= m->partials_cap) return AFD_OK;
  invalidate_graphs(m);
  dfree(m->partials);
  TRY(dalloc(&m->partials, n));
  m->partials_cap = n;
  return AFD_OK;
}

constexpr int TY64 = 8;  // warps per FP64 stencil CTA; the FP32 stencil takes m->ty32 (8 or 16)
// Smallest relative tolerance whose refinement residual is evaluated in double-float arithmetic: its
// rounding, a few 2^-44 of the largest element forces, stays about 1e-12 of ||f|| on voided meshes.
constexpr double RESIDUAL_DF_MIN_TOL = 1e-10;

static void geom32(const Grid& g, int ty, int kz, int& tiles_x, dim3& grid) {
  if (ty == 8)
    StencilGeom2<8>::get(g, kz, tiles_x, grid);
  else
    StencilGeom2<16>::get(g, kz, tiles_x, grid);
}

static void geom3(const Grid& g, int ty, int kz, bool rp, int& tiles_x, dim3& grid) {
  int tiles_y;
  if (ty == 8)
    rp ? St3Geom<8, true>::get(g, kz, tiles_x, tiles_y, grid) : St3Geom<8>::get(g, kz, tiles_x, tiles_y, grid);
  else
    rp ? St3Geom<16, true>::get(g, kz, tiles_x, tiles_y, grid) : St3Geom<16>::get(g, kz, tiles_x, tiles_y, grid);
}

// The FP32 stencil runs load cases in pairs (packed-band kernel, pair mode)
// when the autotuner chose it for this mesh and there are at least two.
static bool use_rp(const afd_mesh* m, int nrhs) { return m->rp32 && m->async32 == 2 && nrhs >= 2; }

static void stencil_geom(const afd_mesh* m, bool f64, int& tiles_x, dim3& grid, int nrhs = 1) {
  if (f64)
    StencilGeom<TY64>::get(m->gr, m->kz, tiles_x, grid);
  else if (m->async32 == 2)
    geom3(m->gr, m->ty32, m->kz32, use_rp(m, nrhs), tiles_x, grid);
  else
    geom32(m->gr, m->ty32, m->kz32, tiles_x, grid);
}

// Per-tile flags of the packed-band stencil for the current supports, CTA
// height and mode (recomputed when any changes).
static int ensure_tile_flags(afd_mesh* m, bool rp) {
  const int key = 2 * m->ty32 + (rp ? 1 : 0);
  if (m->tflags_ty == key && m->tflags) return AFD_OK;
  int tx;
  dim3 grid;
  geom3(m->gr, m->ty32, 1, rp, tx, grid);
  const size_t nt = grid.x;
  if (nt > m->tflags_cap) {
    dfree(m->tflags);
    m->tflags_cap = 0;
    TRY(dalloc(&m->tflags, nt));
    m->tflags_cap = nt;
  }
  if (m->ty32 == 8)
    rp ? k_st3_tile_flags<8, true><<<(unsigned)nt, 256, 0, m->s>>>(m->gr, m->fixed, tx, m->tflags)
       : k_st3_tile_flags<8, false><<<(unsigned)nt, 256, 0, m->s>>>(m->gr, m->fixed, tx, m->tflags);
  else
    rp ? k_st3_tile_flags<16, true><<<(unsigned)nt, 256, 0, m->s>>>(m->gr, m->fixed, tx, m->tflags)
       : k_st3_tile_flags<16, false><<<(unsigned)nt, 256, 0, m->s>>>(m->gr, m->fixed, tx, m->tflags);
  m->launches++;
  CK(cudaGetLastError());
  m->tflags_ty = key;
  return AFD_OK;
}


static int stencil_blocks(const afd_mesh* m, bool f64, int nrhs = 1) {
  int tx;
  dim3 g;
  stencil_geom(m, f64, tx, g, nrhs);
  return (int)(g.x * g.y);
}

// Kernels that need more than the default 48 KB of dynamic shared memory get
// their attribute raised once per device (the attribute is per device; meshes
// of one process may live on several, and server workers launch from several
// threads).  bit: which kernel.
static std::atomic<unsigned long long> g_optin[64];
template <typename F>
static int opt_in_once(int bit, F&& set) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(AFD_ERR_INVALID_ARG, "device index %d out of range", dev);
  const unsigned long long mask = 1ull << bit;
  if (g_optin[dev].load(std::memory_order_acquire) & mask) return AFD_OK;
  CK(set());
  g_optin[dev].fetch_or(mask, std::memory_order_acq_rel);
  return AFD_OK;
}

template <int TY, int MODE>
static int launch_st3(afd_mesh* m, const StencilArgs<float, float>& a, dim3 grid, int nrhs) {
  const size_t dyn = st3_smem_bytes<TY, MODE>();
  if (use_rp(m, nrhs)) {
    if (a.counter) return fail(AFD_ERR_INVALID_ARG, "load-case pairs take no last-CTA step length");
    TRY(opt_in_once(32 + 2 * MODE + (TY == 8 ? 0 : 1), [&]() {
      return cudaFuncSetAttribute(st3_kernel<TY, MODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    }));
    grid.z = (nrhs + 1) / 2;
    CK(launch_ex(m->pdl_now, st3_kernel<TY, MODE, true>, grid, dim3(ST_TX * TY), dyn, m->s, a,
                 (const uint8_t*)m->tflags, nrhs));
    return AFD_OK;
  }
  TRY(opt_in_once(24 + 2 * MODE + (TY == 8 ? 0 : 1), [&]() {
    return cudaFuncSetAttribute(st3_kernel<TY, MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  }));
  CK(launch_ex(m->pdl_now, st3_kernel<TY, MODE, false>, grid, dim3(ST_TX * TY), dyn, m->s, a,
               (const uint8_t*)m->tflags, nrhs));
  return AFD_OK;
}

template <typename T, int MODE, typename TF, typename C = T>
static int launch_stencil(afd_mesh* m, const T* u, T* y, const T* E, const TF* f, float* y32, double* partials,
                          const int* done, int nrhs, const ElemConsts<T>& K, CGState* st = nullptr,
                          unsigned int* counter = nullptr, const T* z = nullptr, const double* mu = nullptr,
                          T* pout = nullptr, const IterPartials* ip = nullptr) {
  constexpr bool F64 = sizeof(T) == 8;
  StencilArgs<T, TF> a;
  a.gr = m->gr;
  a.u = u;
  a.y = y;
  a.E = E;
  a.fixed = m->fixed;
  a.K = K;
  a.f = f;
  a.y32 = y32;
  a.partials = partials;
  a.done = done;
  a.kz = F64 ? m->kz : m->kz32;
  a.st = st;
  a.counter = counter;
  a.z = z;
  a.mu = mu;
  a.pout = pout;
  a.gp = m->gp;
  a.ip = ip ? *ip : IterPartials{nullptr, 0, nullptr, 0, 0};
  dim3 grid;
  stencil_geom(m, F64, a.tiles_x, grid, nrhs);
  grid.z = nrhs;
  if constexpr (F64) {
    CK(launch_ex(m->pdl_now, stencil_kernel<T, TY64, MODE, TF, C>, grid, dim3(ST_TX * TY64), 0, m->s, a));
  } else {
    static_assert(std::is_same<TF, float>::value, "the FP32 stencil takes FP32 right-hand sides");
    // the packed FP32 kernel forms p in ST_APPLY_DOT only, and always there
    if ((MODE == ST_APPLY_DOT) != (z != nullptr)) return fail(AFD_ERR_INVALID_ARG, "stencil mode / z mismatch");
    if (m->async32 == 2) {
      TRY(ensure_tile_flags(m, use_rp(m, nrhs)));
      if (m->ty32 == 8)
        TRY((launch_st3<8, MODE>(m, a, grid, nrhs)));
      else
        TRY((launch_st3<16, MODE>(m, a, grid, nrhs)));
    } else if (m->async32) {   // the asynchronous staging ring lives in dynamic shared memory
      const int ti = m->ty32 == 8 ? 0 : 1;
      const size_t dyn =
          (m->ty32 == 8 ? stencil2_ring_floats<8, MODE>() : stencil2_ring_floats<16, MODE>()) * sizeof(float);
      TRY(opt_in_once(2 * MODE + ti, [&]() {
        return m->ty32 == 8
                   ? cudaFuncSetAttribute(stencil2_kernel<8, MODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn)
                   : cudaFuncSetAttribute(stencil2_kernel<16, MODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      }));
      if (m->ty32 == 8)
        CK(launch_ex(m->pdl_now, stencil2_kernel<8, MODE, true>, grid, dim3(ST_TX * 8), dyn, m->s, a));
      else
        CK(launch_ex(m->pdl_now, stencil2_kernel<16, MODE, true>, grid, dim3(ST_TX * 16), dyn, m->s, a));
    } else {
      if (m->ty32 == 8)
        CK(launch_ex(m->pdl_now, stencil2_kernel<8, MODE, false>, grid, dim3(ST_TX * 8), 0, m->s, a));
      else
        CK(launch_ex(m->pdl_now, stencil2_kernel<16, MODE, false>, grid, dim3(ST_TX * 16), 0, m->s, a));
    }
  }
  m->launches++;
  CK(cudaGetLastError());
  return AFD_OK;
}

static int pick_group(int nx, int ny, int nz, int req) {
  if (req > 0) return req;
  for (int g = 4; g <= 1024; g *= 2) {
    long ng = (long)std::max(nx / g, 1) * std::max(ny / g, 1) * std::max(nz / g, 1);
    if (6 * ng <= 3072) return g;
  }
  return 1024;
}

template <typename T>
static int ensure_work(afd_mesh* m, Work<T>& w, int nrhs) {
  if (w.cap >= nrhs) return AFD_OK;
  invalidate_graphs(m);
  dfree(w.x); dfree(w.r); dfree(w.z); dfree(w.p); dfree(w.q); dfree(w.t); dfree(w.b); dfree(w.r2);
  if (w.graph) { cudaGraphExecDestroy(w.graph); w.graph = nullptr; }
  const size_t n = (size_t)nrhs * m->gr.vs;
  TRY(dalloc(&w.x, n)); TRY(dalloc(&w.r, n)); TRY(dalloc(&w.z, n)); TRY(dalloc(&w.p, n));
  TRY(dalloc(&w.q, n)); TRY(dalloc(&w.t, n)); TRY(dalloc(&w.b, n)); TRY(dalloc(&w.r2, n));
  w.cap = nrhs;
  return AFD_OK;
}

static int ensure_rhs(afd_mesh* m, int nrhs) {
  if (m->cap >= nrhs) return AFD_OK;
  invalidate_graphs(m);
  dfree(m->f64); dfree(m->u64); dfree(m->st); dfree(m->done); dfree(m->v); dfree(m->mu); dfree(m->wr);
  dfree(m->fbuf);
  const size_t n = (size_t)nrhs * m->gr.vs;
  TRY(dalloc(&m->f64, n)); TRY(dalloc(&m->u64, n));
  TRY(dalloc(&m->st, (size_t)nrhs)); TRY(dalloc(&m->done, (size_t)nrhs));
  TRY(dalloc(&m->v, (size_t)nrhs * m->nc)); TRY(dalloc(&m->mu, (size_t)nrhs * m->nc));
  TRY(dalloc(&m->wr, (size_t)nrhs * m->nc));
  dfree(m->cpart); dfree(m->grec); dfree(m->gcount); dfree(m->upart);
  m->cpart_cap = (size_t)nrhs * m->gp.ng * m->nsplit * 12;
  TRY(dalloc(&m->cpart, m->cpart_cap));
  TRY(dalloc(&m->grec, (size_t)nrhs * m->gp.ng * 12));
  TRY(dalloc(&m->upart, (size_t)nrhs * RED_BLOCKS * 2));
  TRY(dalloc(&m->gcount, (size_t)nrhs * m->gp.ng));
  CK(cudaMemsetAsync(m->gcount, 0, (size_t)nrhs * m->gp.ng * sizeof(unsigned int), m->s));
  TRY(dalloc(&m->fbuf, (size_t)nrhs * m->gr.nelem));
  m->cap = nrhs;
  // graphs captured for a smaller RHS count stay valid; none need freeing here
  return AFD_OK;
}

// ---------------------------------------------------------------------------
// coarse problem
// ---------------------------------------------------------------------------
// In-place inverse of the SPD coarse matrix A (nc x nc, type T) by blocked
// Gauss-Jordan sweeps; a relative pivot below `rel` means W^T K W is singular.
template <typename T>
static int invert_coarse(afd_mesh* m, T* A, double rel) {
  const int nc = m->nc;
  // A holds the unit-diagonal scaled matrix: pivots are tested against 1
  const double one = 1.0;
  CK(cudaMemcpyAsync(m->dmax, &one, sizeof(double), cudaMemcpyHostToDevice, m->s));
  CK(cudaMemsetAsync(m->dstatus, 0, sizeof(int), m->s));
  T* P = (T*)m->gjP;
  T* B = (T*)m->gjB;
  T* R = (T*)m->gjR;
  const dim3 ug((nc + 31) / 32, (nc + 31) / 32);
  // The 3 launches per panel of GJ_NB columns are a few microseconds each: they
  // are captured once per mesh and type into a graph (A, the scratch and the
  // tolerance do not change for the mesh's life) and replayed.
  const int npanel = (nc + GJ_NB - 1) / GJ_NB;
  cudaGraphExec_t& gx = m->gj_graph[sizeof(T) == 8 ? 1 : 0];
  if (!gx) {
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(m->s, cudaStreamCaptureModeThreadLocal));
    for (int k0 = 0; k0 < nc; k0 += GJ_NB) {
      const int nb = std::min(GJ_NB, nc - k0);
      k_gj_pivot<T><<<1, 32, 0, m->s>>>(A, nc, k0, P, m->dmax, rel, m->dstatus);
      k_gj_panel<T><<<(nc * nb + 255) / 256, 256, 0, m->s>>>(A, nc, k0, P, B, R);
      k_gj_update<T><<<ug, 256, 0, m->s>>>(A, nc, k0, P, B, R, k0 + GJ_NB >= nc ? 1 : 0);
    }
    k_unscale_dense<T><<<grid_blocks((size_t)nc * nc, 256, 4096), 256, 0, m->s>>>(nc, m->gjD, A);
    const cudaError_t le = cudaGetLastError();
    const cudaError_t ce = cudaStreamEndCapture(m->s, &graph);
    if (le != cudaSuccess) return fail(AFD_ERR_CUDA, "coarse inverse capture: %s", cudaGetErrorString(le));
    if (ce != cudaSuccess) return fail(AFD_ERR_CUDA, "coarse inverse capture: %s", cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&gx, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      gx = nullptr;
      return fail(AFD_ERR_CUDA, "coarse inverse graph: %s", cudaGetErrorString(ie));
    }
  }
  CK(cudaGraphLaunch(gx, m->s));
  m->launches += 3 * npanel + 1;
  int status = 0;
  CK(cudaMemcpyAsync(&status, m->dstatus, sizeof(int), cudaMemcpyDeviceToHost, m->s));
  CK(cudaStreamSynchronize(m->s));
  if (status != 0)
    return fail(AFD_ERR_COARSE_SINGULAR, "coarse matrix W^T K W is singular (are there enough supports?)");
  return AFD_OK;
}

// A = Ec^{-1} in type T: the unit-diagonal scaled matrix, inverted by the
// blocked Gauss-Jordan sweeps and unscaled.
template <typename T>
static int scale_and_invert(afd_mesh* m, T* A, double rel) {
  const size_t nn = (size_t)m->nc * m->nc;
  k_diag_rsqrt<<<grid_blocks((size_t)m->nc, 256, 64), 256, 0, m->s>>>(m->nc, m->Ec, m->gjD); m->launches++;
  k_scale_dense<T><<<grid_blocks(nn, 256, 4096), 256, 0, m->s>>>(m->nc, m->Ec, m->gjD, A); m->launches++;
  return invert_coarse<T>(m, A, rel);
}

// E = W^T K W into m->Ec (FP64 sums; element math in FP32 on the mixed path).
static int assemble_coarse(afd_mesh* m) {
  if (!m->has_moduli) return fail(AFD_ERR_STATE, "moduli not set");
  const int nc = m->nc;
  const size_t nn = (size_t)nc * nc;
  if (!m->Ec) {
    TRY(dalloc(&m->Ec, nn));
    TRY(dalloc(&m->gjP, (size_t)GJ_NB * GJ_NB));
    TRY(dalloc(&m->gjD, (size_t)nc));
    TRY(dalloc(&m->gjB, (size_t)nc * GJ_NB));
    TRY(dalloc(&m->gjR, (size_t)nc * GJ_NB));
    TRY(dalloc(&m->dmax, 1));
    TRY(dalloc(&m->dstatus, 1));
  }
  CK(cudaMemsetAsync(m->Ec, 0, nn * sizeof(double), m->s));
  if (m->cut) {
    // from the cut-element records: E_GG in nself shares, the 13 neighbours after G with their transposes
    const int nself = std::max(1, std::min(16, m->gp.g / 2));
    const size_t need = (size_t)m->gp.ng * nself * 36;
    if (need > m->cpart_c_cap) {
      dfree(m->cpart_c);
      m->cpart_c_cap = 0;
      TRY(dalloc(&m->cpart_c, need));
      m->cpart_c_cap = need;
    }
    if (!m->ccount) {
      TRY(dalloc(&m->ccount, (size_t)m->gp.ng));
      CK(cudaMemsetAsync(m->ccount, 0, (size_t)m->gp.ng * sizeof(unsigned int), m->s));
    }
    const dim3 cg(m->gp.ng, nself + 13);
    if (m->opt.coarse_fp64)
      k_coarse_cut<double><<<cg, COARSE_THREADS, 0, m->s>>>(m->gr, m->gp, nself, m->cut, m->cut_off, m->E64,
                                                             m->w64.K, m->Ec, m->cpart_c, m->ccount);
    else
      k_coarse_cut<float><<<cg, COARSE_THREADS, 0, m->s>>>(m->gr, m->gp, nself, m->cut, m->cut_off, m->E64,
                                                            m->w32.K, m->Ec, m->cpart_c, m->ccount);
    m->launches++;
    CK(cudaGetLastError());
    return AFD_OK;
  }
  const dim3 grid(m->gp.ng, 27);
  if (m->opt.precision == AFD_FP64 || m->opt.coarse_fp64) {
    k_coarse_block<double><<<grid, COARSE_THREADS, 0, m->s>>>(m->gr, m->gp, m->E64, m->fixed, m->w64.K, m->Ec); m->launches++;
  } else {
    k_coarse_block<float><<<grid, COARSE_THREADS, 0, m->s>>>(m->gr, m->gp, m->E64, m->fixed, m->w32.K, m->Ec); m->launches++;
  }
  CK(cudaGetLastError());
  return AFD_OK;
}

// K W on the groups' node shells for the work type of the solve.
template <typename T>
static int build_aw(afd_mesh* m, Work<T>& w) {
  if (!m->has_loads) return fail(AFD_ERR_STATE, "supports not set");
  if (w.aw_cap < m->aw_total) {
    invalidate_graphs(m);
    dfree(w.AW);
    TRY(dalloc(&w.AW, m->aw_total));
    w.aw_cap = m->aw_total;
  }
  const dim3 grid(m->gp.ng, m->nsplit_aw);
  k_build_aw<T><<<grid, 128, 0, m->s>>>(m->gr, m->gp, m->nsplit_aw, m->E64, m->fixed, m->gbox, m->aw_off, w.K, w.AW,
                                         m->aw_node); m->launches++;
  CK(cudaGetLastError());
  return AFD_OK;
}

// The FP32 graph path forms (K W)^T z from the cut elements of each group;
// the FP64 path and the persistent kernel read K W stored on the node shells.
static bool uses_stored_aw(const afd_mesh* m) { return m->opt.precision == AFD_FP64 || m->opt.persistent; }

// The cut-element records of the FP32 graph path (k_build_cut_recs), rebuilt
// with the supports; left null (the kernel decodes each element's position
// instead) when a group is too wide for their 10-bit coordinates.
static int build_cut_records(afd_mesh* m) {
  if (uses_stored_aw(m)) return AFD_OK;
  const Grid& g = m->gr;
  const Groups& gp = m->gp;
  std::vector<long long> off(gp.ng + 1);
  size_t tot = 0;
  bool fits = true;
  for (int G = 0; G < gp.ng; ++G) {
    int b[12];
    elem_shell_bounds(g, gp, G, m->gbox_h.data() + 6 * G, b);
    Shell sh;
    sh.init(b[0], b[1], b[2], b[3], b[4], b[5], b[6], b[7], b[8], b[9], b[10], b[11], false);
    for (int d = 0; d < 3; ++d) fits = fits && b[2 * d + 1] - b[2 * d] + 2 <= 1023;
    off[G] = (long long)tot;
    tot += (size_t)sh.count;
  }
  off[gp.ng] = (long long)tot;
  invalidate_graphs(m);
  if (!fits) {
    dfree(m->cut);
    m->cut = nullptr;
    m->cut_cap = 0;
    return AFD_OK;
  }
  if (!m->cut_off) TRY(dalloc(&m->cut_off, (size_t)gp.ng + 1));
  if (tot > m->cut_cap || !m->cut) {
    dfree(m->cut);
    m->cut = nullptr;
    m->cut_cap = 0;
    TRY(dalloc(&m->cut, std::max<size_t>(tot, 1)));
    m->cut_cap = tot;
  }
  CK(cudaMemcpyAsync(m->cut_off, off.data(), (gp.ng + 1) * sizeof(long long), cudaMemcpyHostToDevice, m->s));
  k_build_cut_recs<<<gp.ng, 256, 0, m->s>>>(g, gp, m->fixed, m->gbox, m->cut_off, m->cut); m->launches++;
  CK(cudaGetLastError());
  return AFD_OK;
}

template <typename T>
static int launch_coarse_rhs(afd_mesh* m, Work<T>& w, int nsplit, int nrhs, bool pdl) {
  const dim3 ug(m->gp.ng, nsplit, nrhs);
  if (sizeof(T) == 4 && !uses_stored_aw(m))
    CK(launch_ex(pdl, k_coarse_rhs_cut<T>, ug, dim3(256), 0, m->s, m->gr, m->gp, nsplit, (const T*)w.r,
                 (const T*)w.z, (const T*)w.E, (const uint8_t*)m->fixed, (const int*)m->gbox, w.K, m->cpart, m->grec,
                 m->gcount, (const CGState*)m->st, (const uint4*)m->cut, (const long long*)m->cut_off));
  else
    CK(launch_ex(pdl, k_coarse_rhs<T>, ug, dim3(256), 0, m->s, m->gr, m->gp, nsplit, (const T*)w.r, (const T*)w.z,
                 (const long long*)m->aw_off, (const int*)m->aw_node, (const T*)w.AW, m->cpart, m->grec, m->gcount,
                 (const CGState*)m->st));
  m->launches++;
  return AFD_OK;
}

static int build_coarse(afd_mesh* m) {
  if (m->coarse_valid) return AFD_OK;
  TRY(assemble_coarse(m));
  if (m->opt.precision == AFD_FP64) TRY(build_aw<double>(m, m->w64));
  else if (uses_stored_aw(m)) TRY(build_aw<float>(m, m->w32));
  const size_t nn = (size_t)m->nc * m->nc;
  if (m->opt.precision == AFD_FP64) {
    if (!m->Einv64) TRY(dalloc(&m->Einv64, nn));
    TRY(scale_and_invert<double>(m, m->Einv64, 1e-12));
  } else if (m->opt.coarse_fp64) {
    // FP64 inverse, rounded once to FP32 for the inner iterations' coarse step
    if (!m->Einv64) TRY(dalloc(&m->Einv64, nn));
    if (!m->Einv32) TRY(dalloc(&m->Einv32, nn));
    TRY(scale_and_invert<double>(m, m->Einv64, 1e-12));
    k_convert_dense<float><<<grid_blocks(nn, 256, 4096), 256, 0, m->s>>>(nn, m->Einv64, m->Einv32); m->launches++;
  } else {
    if (!m->Einv32) TRY(dalloc(&m->Einv32, nn));
    TRY(scale_and_invert<float>(m, m->Einv32, 1e-6));
  }
  m->coarse_valid = true;
  return AFD_OK;
}

static int ensure_cpart(afd_mesh* m, int nsplit) {
  const size_t need = (size_t)std::max(m->cap, 1) * m->gp.ng * nsplit * 12;
  if (need <= m->cpart_cap) return AFD_OK;
  invalidate_graphs(m);
  dfree(m->cpart);
  m->cpart_cap = 0;
  TRY(dalloc(&m->cpart, need));
  m->cpart_cap = need;
  return AFD_OK;
}

// Dynamic shared memory of k_coarse_step<T> (v staged in the inverse's type),
// opted in above the 48 KB default once per type; a coarse problem whose v
// does not fit in a CTA's shared memory is refused.
template <typename T>
static int coarse_step_smem(const afd_mesh* m, size_t& bytes) {
  bytes = (size_t)m->nc * sizeof(T);
  constexpr size_t kMax = 200 * 1024;
  if (bytes > kMax)
    return fail(AFD_ERR_INVALID_ARG, "coarse problem too large for the dense inverse (6 x groups above 25600 for FP64, "
                                     "51200 for mixed): use a larger group");
  if (bytes > 40 * 1024)
    TRY(opt_in_once(16 + (sizeof(T) == 8 ? 1 : 0), [&]() {
      return cudaFuncSetAttribute(k_coarse_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMax);
    }));
  return AFD_OK;
}

// Stencil autotuner: the FP32 stencil's variant (stencil2 with register
// prefetch or a cp.async ring, or the packed-band stencil3), CTA shape (8 or
// 16 warps, i.e. 14 or 30 finished node rows) and z depth trade redundant
// halo rows and element layers against the number of CTAs (waves over the
// SMs).  Each candidate is timed as the inner iteration runs it (the fused
// search-direction kernel) on the solver's stream with CUDA events (3
// launches after one warm-up); the fastest is kept for the mesh.
// One fused in-iteration stencil launch for R load cases on zero vectors (the
// autotuner's timed kernel; its cost does not depend on the values).
static int fused_for_tuning(afd_mesh* m, int R) {
  return launch_stencil<float, ST_APPLY_DOT, float>(m, m->w32.p, m->w32.q, m->w32.E, nullptr, nullptr, m->partials,
                                                    nullptr, R, m->w32.K, m->st, nullptr, m->w32.z, m->mu, m->w32.t,
                                                    nullptr);
}

static int autotune_stencil(afd_mesh* m) {
  const int R = std::max(1, m->nrhs);
  TRY(ensure_work(m, m->w32, R));
  const Grid& g = m->gr;
  static const int all_kz[] = {2, 3, 4, 5, 6, 8, 12, 16, 24, 32};
  static const int all_ty[] = {8, 16};
  // a shape the caller pinned (opt.stencil_warps / stencil_planes) is kept
  const std::vector<int> cand_kz = m->opt.stencil_planes ? std::vector<int>{m->kz32}
                                                         : std::vector<int>(all_kz, all_kz + 10);
  const std::vector<int> cand_ty = m->opt.stencil_warps ? std::vector<int>{m->opt.stencil_warps}
                                                        : std::vector<int>(all_ty, all_ty + 2);
  size_t maxp = 0;
  for (int ty : cand_ty)
    for (int kz : cand_kz) {
      int tx;
      dim3 gr;
      geom32(g, ty, kz, tx, gr);
      maxp = std::max(maxp, (size_t)gr.x * gr.y);
      geom3(g, ty, kz, false, tx, gr);
      maxp = std::max(maxp, (size_t)gr.x * gr.y);
      geom3(g, ty, kz, true, tx, gr);
      maxp = std::max(maxp, (size_t)gr.x * gr.y);
    }
  TRY(ensure_partials(m, (size_t)std::max(m->cap, 1) * std::max(maxp, (size_t)2 * RED_BLOCKS)));
  // the timed kernel is the inner iteration's fused one (p = z + W mu + beta p_old, q = K p, p.q) on
  // zero vectors and a zero coarse vector (its cost does not depend on the values)
  CK(cudaMemsetAsync(m->w32.p, 0, (size_t)R * g.vs * sizeof(float), m->s));
  CK(cudaMemsetAsync(m->w32.z, 0, (size_t)R * g.vs * sizeof(float), m->s));
  CK(cudaMemsetAsync(m->mu, 0, (size_t)R * m->nc * sizeof(double), m->s));
  CK(cudaMemsetAsync(m->st, 0, (size_t)R * sizeof(CGState), m->s));
  m->rp32 = 0;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_kz = m->kz32, best_ty = m->ty32, best_as = m->async32;
  for (int as = 0; as < 3; ++as)
  for (int ty : cand_ty)
    for (int kz : cand_kz) {
      if (kz > g.nnz && kz != cand_kz.front()) continue;
      m->ty32 = ty;
      m->kz32 = kz;
      m->async32 = as;
      auto fused = [&]() { return fused_for_tuning(m, 1); };
      TRY(fused());
      CK(cudaEventRecord(e0, m->s));
      for (int rep = 0; rep < 3; ++rep) TRY(fused());
      CK(cudaEventRecord(e1, m->s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_kz = kz;
        best_ty = ty;
        best_as = as;
      }
    }
  m->kz32 = best_kz;
  m->ty32 = best_ty;
  m->async32 = best_as;
  if (R >= 2) {
    // several load cases: the packed-band kernel with the cases in pairs against the best single-case
    // variant launched for all of them (both for the R cases of this mesh)
    auto time_r = [&](float& ms) -> int {
      TRY(fused_for_tuning(m, R));
      CK(cudaEventRecord(e0, m->s));
      for (int rep = 0; rep < 3; ++rep) TRY(fused_for_tuning(m, R));
      CK(cudaEventRecord(e1, m->s));
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&ms, e0, e1));
      return AFD_OK;
    };
    float best_r = 0.f;
    TRY(time_r(best_r));
    int rp_ty = 0, rp_kz = 0;
    for (int ty : cand_ty)
      for (int kz : cand_kz) {
        if (kz > g.nnz && kz != cand_kz.front()) continue;
        m->ty32 = ty;
        m->kz32 = kz;
        m->async32 = 2;
        m->rp32 = 1;
        float ms = 0.f;
        TRY(time_r(ms));
        if (ms < best_r) {
          best_r = ms;
          rp_ty = ty;
          rp_kz = kz;
        }
      }
    if (rp_ty) {
      m->ty32 = rp_ty;
      m->kz32 = rp_kz;
      m->async32 = 2;
      m->rp32 = 1;
    } else {
      m->kz32 = best_kz;
      m->ty32 = best_ty;
      m->async32 = best_as;
      m->rp32 = 0;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->tuned = true;
  invalidate_graphs(m);  // captured launches bake in the grid
  return AFD_OK;
}

// Shares per group of the coarse right-hand side: fewer shares amortise the
// per-block 12-value reduction, more shares shorten each block's load chain.
// Timed like the stencil (3 launches after one warm-up, one RHS, FP32) on the
// mesh's own shells; needs the coarse data (build_coarse) in place.
static int autotune_coarse_split(afd_mesh* m) {
  TRY(ensure_work(m, m->w32, 1));
  const Grid& g = m->gr;
  static const int cand[] = {1, 2, 3, 4, 6, 8, 12, 16};
  CK(cudaMemsetAsync(m->w32.r, 0, (size_t)g.vs * sizeof(float), m->s));
  CK(cudaMemsetAsync(m->w32.z, 0, (size_t)g.vs * sizeof(float), m->s));
  CGState st0;
  memset(&st0, 0, sizeof(st0));
  CK(cudaMemcpyAsync(m->st, &st0, sizeof(CGState), cudaMemcpyHostToDevice, m->s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_ns = m->nsplit;
  for (int ns : cand) {
    if (ns > m->gp.g) break;
    TRY(ensure_cpart(m, ns));
    for (int rep = 0; rep < 4; ++rep) {
      if (rep == 1) CK(cudaEventRecord(e0, m->s));
      TRY(launch_coarse_rhs<float>(m, m->w32, ns, 1, false));
    }
    CK(cudaEventRecord(e1, m->s));
    CK(cudaEventSynchronize(e1));
    CK(cudaGetLastError());
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      best_ns = ns;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  m->nsplit = best_ns;
  invalidate_graphs(m);
  return AFD_OK;
}


// ---------------------------------------------------------------------------
// FP32 inner DPCG iterations as one cooperative persistent kernel
// (dpcg_persistent.cuh).  Launched after the deflated start; returns with
// *launched = 0 (and nothing enqueued) when the device cannot co-schedule the
// grid, in which case the caller runs the CUDA-graph path.
// ---------------------------------------------------------------------------
template <int TY>
static int launch_persistent(afd_mesh* m, Work<float>& w, float* x, int nrhs, int& launched) {
  launched = 0;
  const Grid& gr = m->gr;
  int nsm = 0, coop = 0;
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, m->device));
  if (!coop || nrhs > PERSIST_MAX_RHS) return AFD_OK;
  const size_t smem = (size_t)m->nc * sizeof(double);
  if (smem > 48 * 1024)
    CK(cudaFuncSetAttribute(k_dpcg_persistent<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dpcg_persistent<TY>, ST_TX * TY, smem));
  if (per_sm < 1) return AFD_OK;
  const int nb = per_sm * nsm;
  PersistArgs pa;
  memset(&pa, 0, sizeof(pa));
  pa.sa.gr = gr;
  pa.sa.E = w.E;
  pa.sa.fixed = m->fixed;
  pa.sa.K = w.K;
  pa.sa.kz = m->kz32;
  pa.sa.gp = m->gp;
  dim3 sg;
  StencilGeom2<TY>::get(gr, m->kz32, pa.sa.tiles_x, sg);
  pa.ntiles = (int)(sg.x * sg.y);
  pa.nrhs = nrhs;
  pa.x = x;
  pa.r = w.r;
  pa.z = w.z;
  pa.q = w.q;
  pa.P0 = w.p;
  pa.P1 = w.t;
  pa.invd = w.invd;
  pa.nc = m->nc;
  pa.nsplit = std::max(1, std::min(m->gp.g, nb / std::max(1, m->gp.ng)));
  pa.aw_off = m->aw_off;
  pa.aw_node = m->aw_node;
  pa.AW = w.AW;
  pa.Einv = m->Einv32;
  pa.mu = m->mu;
  // tile partials, then the per-CTA records (4 doubles each, 32-byte aligned for the vector loads)
  const size_t st_len = ((size_t)nrhs * pa.ntiles + 3) / 4 * 4;
  const size_t need = st_len + (size_t)nrhs * 4 * (size_t)nb;
  if (need > m->ppart_cap) {
    dfree(m->ppart);
    m->ppart_cap = 0;
    TRY(dalloc(&m->ppart, need));
    m->ppart_cap = need;
  }
  const size_t needr = (size_t)nrhs * m->gp.ng * pa.nsplit * 12;
  if (needr > m->prec_cap) {
    dfree(m->prec);
    m->prec_cap = 0;
    TRY(dalloc(&m->prec, needr));
    m->prec_cap = needr;
  }
  if (!m->gbar) TRY(dalloc(&m->gbar, 1));
  if (!m->ptime) {
    TRY(dalloc(&m->ptime, 10));
    CK(cudaMemsetAsync(m->ptime, 0, 10 * sizeof(unsigned long long), m->s));
  }
  pa.ptime = m->ptime;
  pa.rec = m->prec;
  pa.part_st = m->ppart;
  pa.part_up = m->ppart + st_len;
  pa.st = m->st;
  pa.done = m->done;
  pa.bar = m->gbar;
  CK(cudaMemsetAsync(m->gbar, 0, sizeof(GridBarrier), m->s));
  void* args[] = {&pa};
  CK(cudaLaunchCooperativeKernel((const void*)k_dpcg_persistent<TY>, dim3(nb), dim3(ST_TX * TY), args, smem, m->s));
  m->launches++;
  launched = 1;
  return AFD_OK;
}

// ---------------------------------------------------------------------------
// deflated PCG (Sec. 3.5) in type T on K x = b; x holds the initial guess
// (x_zero: the caller zeroed it, so the first residual is b itself).
// Per-RHS stop: r.r <= target2[r]; RHS with active[r] == 0 are skipped.
// ---------------------------------------------------------------------------
template <typename T, typename TB>
static int dpcg(afd_mesh* m, Work<T>& w, const TB* b, T* x, bool x_zero, int nrhs, const std::vector<double>& target2,
                const std::vector<int>& active, int max_iters, std::vector<CGState>& out) {
  constexpr bool F64 = sizeof(T) == 8;
  const Grid& gr = m->gr;
  const int nsb = stencil_blocks(m, F64, nrhs);
  TRY(ensure_partials(m, (size_t)nrhs * std::max(nsb, 2 * RED_BLOCKS)));
  // state init
  std::vector<CGState> h(nrhs);
  std::vector<int> hd(nrhs);
  for (int r = 0; r < nrhs; ++r) {
    memset(&h[r], 0, sizeof(CGState));
    h[r].target2 = target2[r];
    h[r].max_iters = max_iters;
    h[r].done = active[r] ? 0 : 1;
    h[r].rzs[0] = std::numeric_limits<double>::infinity();   // beta_0 = rho_0 / inf = 0
    hd[r] = h[r].done;
  }
  CK(cudaMemcpyAsync(m->st, h.data(), nrhs * sizeof(CGState), cudaMemcpyHostToDevice, m->s));
  CK(cudaMemcpyAsync(m->done, hd.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, m->s));
  const dim3 gg(m->gp.ng, nrhs);
  const dim3 pg(grid_blocks(gr.nnodes, 256, 4 * RED_BLOCKS), nrhs);
  const int crows = (m->nc * 32 + CSTEP_THREADS - 1) / CSTEP_THREADS;
  size_t csmem = 0;
  TRY(coarse_step_smem<T>(m, csmem));
  const T* Einv = F64 ? (const T*)m->Einv64 : (const T*)m->Einv32;
  unsigned int* cnt_co = m->counters + MAX_RHS;  // coarse step
  T* P[2] = {w.p, w.t};
  const dim3 vg(RED_BLOCKS, nrhs);
  // r = b - K x ; x += W Einv W^T r ; r = b - K x  (deflated start); for x = 0 the first r is b itself
  if constexpr (std::is_same<T, TB>::value) {
    if (x_zero) {
      k_restrict<T><<<gg, 256, 0, m->s>>>(gr, m->gp, b, nullptr, m->fixed, m->v, nullptr, m->st); m->launches++;
    }
  }
  if (!x_zero || !std::is_same<T, TB>::value) {
    TRY((launch_stencil<T, ST_RESIDUAL, TB>(m, x, w.r, w.E, b, nullptr, m->partials, m->done, nrhs, w.K)));
    k_restrict<T><<<gg, 256, 0, m->s>>>(gr, m->gp, w.r, nullptr, m->fixed, m->v, nullptr, m->st); m->launches++;
  }
  k_coarse_solve<T><<<(m->nc * 32 + 255) / 256, 256, 0, m->s>>>(m->nc, nrhs, Einv, m->v, m->mu, m->st); m->launches++;
  k_prolong<T><<<pg, 256, 0, m->s>>>(2, gr, m->gp, x, nullptr, m->mu, m->fixed, m->st); m->launches++;
  TRY((launch_stencil<T, ST_RESIDUAL, TB>(m, x, w.r, w.E, b, nullptr, m->partials, m->done, nrhs, w.K)));
  // Two-level preconditioned residual y = z + W Einv W^T (r - K z), z = M^-1 r
  // (the A-DEF2 form of deflation: the W^T r term keeps W^T r from drifting
  // under rounding, which the plain projected recurrence does not).  The
  // initial step runs the vector update with alpha = 0 (p = q = 0).
  CK(cudaMemsetAsync(P[0], 0, (size_t)nrhs * gr.vs * sizeof(T), m->s));
  CK(cudaMemsetAsync(w.q, 0, (size_t)nrhs * gr.vs * sizeof(T), m->s));
  k_update<T><<<vg, RED_THREADS, 0, m->s>>>(gr.ndof, gr.vs, x, w.r, w.z, P[0], w.q, w.invd, m->upart, m->st, nullptr,
                                            0, m->done); m->launches++;
  TRY(launch_coarse_rhs<T>(m, w, m->nsplit, nrhs, false));
  const size_t ured = (size_t)nrhs * crows * 2;
  if (ured > m->updred_cap) {
    invalidate_graphs(m);
    dfree(m->updred);
    m->updred_cap = 0;
    TRY(dalloc(&m->updred, ured));
    m->updred_cap = ured;
  }
  k_coarse_step<T><<<crows, CSTEP_THREADS, csmem, m->s>>>(m->nc, nrhs, Einv, m->mu, m->st, m->grec, m->wr, 2, m->done, cnt_co,
                                               m->upart, RED_BLOCKS, m->updred); m->launches++;
  CK(cudaGetLastError());

  if constexpr (!F64) {
    if (m->opt.persistent) {
      int launched = 0;
      if (m->ty32 == 8)
        TRY(launch_persistent<8>(m, w, x, nrhs, launched));
      else
        TRY(launch_persistent<16>(m, w, x, nrhs, launched));
      if (launched) {
        out.resize(nrhs);
        CK(cudaMemcpyAsync(out.data(), m->st, nrhs * sizeof(CGState), cudaMemcpyDeviceToHost, m->s));
        CK(cudaStreamSynchronize(m->s));
        for (int r = 0; r < nrhs; ++r)
          if (out[r].status == AFD_ERR_CUDA) return fail(AFD_ERR_CUDA, "persistent solver: a grid-barrier wait ran out");
        return AFD_OK;
      }
    }
  }

  // One chunk of iterations (even length), captured once into a graph.  Per
  // iteration: the stencil forms p = y + beta p_old while applying K to it
  // (and takes alpha), the vector update (x, r, z, r.z, r.r), the coarse
  // right-hand side, the coarse step (mu, beta).
  auto enqueue_chunk = [&]() -> int {
    for (int it = 0; it < m->opt.check_every; ++it) {
      T* pold = P[it & 1];
      T* pnew = P[(it + 1) & 1];
      const IterPartials ip{m->updred, crows, m->wr, crows, it & 1};
      TRY((launch_stencil<T, ST_APPLY_DOT, TB>(m, pold, w.q, w.E, nullptr, nullptr, m->partials, m->done, nrhs, w.K,
                                                m->st, nullptr, w.z, m->mu, pnew, &ip)));
      const bool pdl = m->pdl_now;
      CK(launch_ex(pdl, k_update<T>, vg, dim3(RED_THREADS), 0, m->s, gr.ndof, gr.vs, x, w.r, w.z, (const T*)pnew,
                   (const T*)w.q, (const T*)w.invd, m->upart, m->st, (const double*)m->partials, nsb, m->done));
      m->launches++;
      TRY(launch_coarse_rhs<T>(m, w, m->nsplit, nrhs, pdl));
      CK(launch_ex(pdl, k_coarse_step<T>, dim3(crows), dim3(CSTEP_THREADS), csmem, m->s, m->nc, nrhs, (const T*)Einv, m->mu,
                   m->st, (const double*)m->grec, m->wr, 1, m->done, cnt_co, (const double*)m->upart, (int)RED_BLOCKS,
                   m->updred));
      m->launches++;
    }
    CK(cudaGetLastError());
    return AFD_OK;
  };
  // the graph bakes in x and b; rebuild it when they or the RHS count change
  static_assert(sizeof(void*) == 8, "64-bit");
  cudaGraphExec_t& gexec = w.graph;
  const bool reuse = gexec && w.graph_nrhs == nrhs;
  if (!reuse) {
    if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
    cudaGraph_t graph;
    const int64_t before = m->launches;
    CK(cudaStreamBeginCapture(m->s, cudaStreamCaptureModeThreadLocal));
    m->pdl_now = m->opt.pdl != 0;
    int rc = enqueue_chunk();
    m->pdl_now = false;
    w.graph_kernels = m->launches - before;  // captured, not run
    m->launches = before;
    cudaError_t e = cudaStreamEndCapture(m->s, &graph);
    if (rc != AFD_OK) return rc;
    if (e != cudaSuccess) return fail(AFD_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(AFD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    w.graph_nrhs = nrhs;
  }
  const int max_chunks = max_iters / std::max(1, m->opt.check_every) + 2;
  std::vector<int> flags(nrhs);
  for (int c = 0; c < max_chunks; ++c) {
    CK(cudaMemcpyAsync(flags.data(), m->done, nrhs * sizeof(int), cudaMemcpyDeviceToHost, m->s));
    CK(cudaStreamSynchronize(m->s));
    bool all = true;
    for (int r = 0; r < nrhs; ++r) all &= flags[r] != 0;
    if (all) break;
    CK(cudaGraphLaunch(gexec, m->s));
    m->launches += w.graph_kernels;
  }
  out.resize(nrhs);
  CK(cudaMemcpyAsync(out.data(), m->st, nrhs * sizeof(CGState), cudaMemcpyDeviceToHost, m->s));
  CK(cudaStreamSynchronize(m->s));
  return AFD_OK;
}

// ---------------------------------------------------------------------------
// C ABI (C linkage from the declarations in afd.h)
// ---------------------------------------------------------------------------

void afd_default_options(afd_options* o) {
  if (!o) return;
  o->precision = AFD_MIXED;
  o->group = 0;
  o->nu = 0.3;
  o->h = 1.0;
  o->e_void = 1e-3;
  o->max_iter = 20000;
  o->max_refine = 12;
  o->inner_tol = 2e-5;
  o->check_every = 16;
  o->autotune = 1;
  o->persistent = 0;
  o->stencil_warps = 0;
  o->stencil_planes = 0;
  o->pdl = 0;
  o->inner_aim = 0.7;
  o->coarse_fp64 = 0;
  o->residual_fp64 = 0;
}

const char* afd_last_error(void) { return g_err.c_str(); }

int64_t afd_ndof(const afd_mesh* m) { return m ? m->gr.ndof : 0; }
int64_t afd_nelem(const afd_mesh* m) { return m ? m->gr.nelem : 0; }

int afd_create_mesh(int nx, int ny, int nz, const afd_options* opt, void* cuda_stream, afd_mesh** out) {
  if (!out) return fail(AFD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail(AFD_ERR_INVALID_ARG, "mesh sizes must be >= 1");
  const double nn = (double)(nx + 1) * (ny + 1) * (nz + 1);
  if (3.0 * nn >= 2147483647.0 || (double)nx * ny * nz >= 2147483647.0)
    return fail(AFD_ERR_INVALID_ARG, "mesh too large for 32-bit DOF indices");
  afd_options o;
  afd_default_options(&o);
  if (opt) o = *opt;
  o.check_every += o.check_every & 1;  // p is double-buffered: chunks of even length
  if (!(o.nu > -1.0 && o.nu < 0.5) || !(o.h > 0.0) || !(o.e_void > 0.0) || o.max_iter < 1 || o.max_refine < 0 ||
      o.check_every < 1 || o.group < 0 || (o.precision != AFD_MIXED && o.precision != AFD_FP64) ||
      (o.stencil_warps != 0 && o.stencil_warps != 8 && o.stencil_warps != 16) || o.stencil_planes < 0 ||
      !(o.inner_aim > 0.0 && o.inner_aim < 1.0))
    return fail(AFD_ERR_INVALID_ARG, "invalid options");
  afd_mesh* m = new afd_mesh();
  m->opt = o;
  CK(cudaGetDevice(&m->device));
  m->user = (cudaStream_t)cuda_stream;
  Grid& g = m->gr;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.nnx = nx + 1; g.nny = ny + 1; g.nnz = nz + 1;
  g.nnodes = g.nnx * g.nny * g.nnz;
  g.nelem = nx * ny * nz;
  g.ndof = 3 * g.nnodes;
  g.vs = (g.ndof + 3) / 4 * 4;
  Groups& gp = m->gp;
  gp.g = pick_group(nx, ny, nz, o.group);
  gp.ngx = std::max(nx / gp.g, 1);
  gp.ngy = std::max(ny / gp.g, 1);
  gp.ngz = std::max(nz / gp.g, 1);
  gp.ng = gp.ngx * gp.ngy * gp.ngz;
  gp.h = o.h;
  m->nc = 6 * gp.ng;
  // shares per group of the merged update / coarse right-hand side kernel
  // (about 600 blocks) and of the K W build (about 2400 blocks of 128 threads)
  m->nsplit = std::max(1, std::min(gp.g, (512 + gp.ng - 1) / gp.ng));
  m->nsplit_aw = std::max(1, std::min(16 * gp.g, (2400 + gp.ng - 1) / gp.ng));
  if (m->nc > 8192) {
    delete m;
    return fail(AFD_ERR_INVALID_ARG, "coarse space too large (%d unknowns > 8192): use a larger group", 6 * gp.ng);
  }
  // z planes per CTA before tuning: enough CTAs to fill the GPU a few times
  {
    int tx;
    dim3 gr;
    StencilGeom<TY64>::get(g, g.nnz, tx, gr);
    // about four waves of the FP64 CTAs, at least 4 planes per CTA
    long kz = (long)g.nnz * gr.x / 1216;
    m->kz = (int)std::max(4L, std::min<long>(kz, g.nnz));
    geom32(g, 16, g.nnz, tx, gr);
    // about two waves of 512-thread FP32 CTAs (1 resident per SM)
    kz = (long)g.nnz * gr.x / 304;
    m->kz32 = (int)std::max(4L, std::min<long>(kz, g.nnz));
    if (o.stencil_warps) m->ty32 = o.stencil_warps;
    if (o.stencil_planes) m->kz32 = std::min(o.stencil_planes, g.nnz);
    if (o.stencil_warps && o.stencil_planes) m->tuned = true;   // pinned: nothing to tune
  }
  m->w32.K = make_elem_consts<float>(o.nu, o.h);
  m->w64.K = make_elem_consts<double>(o.nu, o.h);
  int rc = AFD_OK;
  if (cudaStreamCreateWithFlags(&m->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&m->ev, cudaEventDisableTiming) != cudaSuccess) {
    delete m;
    return fail(AFD_ERR_CUDA, "stream creation failed");
  }
  if ((rc = dalloc(&m->E64, (size_t)g.nelem)) != AFD_OK || (rc = dalloc(&m->w32.E, (size_t)g.nelem)) != AFD_OK ||
      (rc = dalloc(&m->w32.invdiag, (size_t)g.nnodes)) != AFD_OK ||
      (rc = dalloc(&m->fixed, (size_t)(g.nnodes + 3) / 4 * 4)) != AFD_OK ||
      (rc = dalloc(&m->w32.invd, (size_t)g.vs)) != AFD_OK ||
      (o.precision == AFD_FP64 && (rc = dalloc(&m->w64.invdiag, (size_t)g.nnodes)) != AFD_OK) ||
      (o.precision == AFD_FP64 && (rc = dalloc(&m->w64.invd, (size_t)g.vs)) != AFD_OK) ||
      (rc = dalloc(&m->fsmall, (size_t)FSMALL_SIZE)) != AFD_OK ||
      (rc = dalloc(&m->counters, (size_t)MAX_RHS + 1)) != AFD_OK ||
      (rc = dalloc(&m->gbox, (size_t)gp.ng * 6)) != AFD_OK ||
      (rc = dalloc(&m->aw_off, (size_t)gp.ng + 1)) != AFD_OK) {
    afd_destroy(m);
    return rc;
  }
  m->w64.E = m->E64;   // the FP64 stencils read the FP64 moduli themselves
  cudaMemsetAsync(m->fixed, 0, (size_t)(g.nnodes + 3) / 4 * 4, m->s);   // padded: read as 4-byte words
  cudaMemsetAsync(m->counters, 0, (MAX_RHS + 1) * sizeof(unsigned int), m->s);
  if (cudaStreamSynchronize(m->s) != cudaSuccess) {
    afd_destroy(m);
    return fail(AFD_ERR_CUDA, "init failed");
  }
  *out = m;
  return AFD_OK;
}

void afd_destroy(afd_mesh* m) {
  if (!m) return;
  DeviceGuard dg(m->device);
  if (m->s) cudaStreamSynchronize(m->s);
  for (auto* wp : {&m->w32}) {
    dfree(wp->x); dfree(wp->r); dfree(wp->z); dfree(wp->p); dfree(wp->q); dfree(wp->t); dfree(wp->b);
    dfree(wp->r2); dfree(wp->AW); dfree(wp->invd);
    dfree(wp->invdiag); dfree(wp->E);
    dfree(m->tflags);
    if (wp->graph) cudaGraphExecDestroy(wp->graph);
  }
  {
    auto* wp = &m->w64;
    dfree(wp->x); dfree(wp->r); dfree(wp->z); dfree(wp->p); dfree(wp->q); dfree(wp->t); dfree(wp->b);
    dfree(wp->r2); dfree(wp->AW); dfree(wp->invd);
    dfree(wp->invdiag);
    wp->E = nullptr;   // the FP64 moduli themselves (E64)
    if (wp->graph) cudaGraphExecDestroy(wp->graph);
  }
  dfree(m->E64); dfree(m->fixed); dfree(m->f64); dfree(m->u64); dfree(m->partials);
  dfree(m->st); dfree(m->done); dfree(m->v); dfree(m->mu); dfree(m->wr); dfree(m->cpart); dfree(m->fbuf); dfree(m->fkeys); dfree(m->kept);
  if (m->sel) cudaFree(m->sel);
  dfree(m->selcnt); dfree(m->fsmall);
  dfree(m->Ec); dfree(m->Einv64); dfree(m->Einv32); dfree(m->gjP); dfree(m->gjB); dfree(m->gjR); dfree(m->gjD);
  for (auto& g : m->gj_graph)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  dfree(m->dmax); dfree(m->dstatus); dfree(m->counters); dfree(m->gbox); dfree(m->aw_off); dfree(m->aw_node);
  dfree(m->cut); dfree(m->cut_off); dfree(m->cpart_c); dfree(m->ccount);
  dfree(m->grec); dfree(m->gcount); dfree(m->upart); dfree(m->updred);
  dfree(m->ppart); dfree(m->prec); dfree(m->gbar); dfree(m->ptime);
  dfree(m->lam64); dfree(m->gadj); dfree(m->dsig); dfree(m->pn_d); dfree(m->lsbuf);
  dfree(m->mX); dfree(m->mmass); dfree(m->mparts);
  dfree(m->mA); dfree(m->mB); dfree(m->mV); dfree(m->mlam); dfree(m->minfo);
  dfree(m->bS6); dfree(m->bcoef);
  for (int q = 0; q < 2; ++q) { dfree(m->lS[q]); dfree(m->lBS[q]); dfree(m->lAS[q]); }
  if (m->ev) cudaEventDestroy(m->ev);
  if (m->s) cudaStreamDestroy(m->s);
  delete m;
}

template <typename T>
__global__ void k_convert(size_t n, const double* __restrict__ a, T* __restrict__ b) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = (T)a[i];
}

// b[d] = a[d / 3]: per-node values repeated for the node's three DOFs.
template <typename T>
__global__ void k_expand3(int ndof, const T* __restrict__ a, T* __restrict__ b) {
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < ndof; d += gridDim.x * blockDim.x) b[d] = a[d / 3];
}

__global__ void k_check_moduli(size_t n, const double* __restrict__ E, int* bad) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!(E[i] > 0.0) || !isfinite(E[i])) *bad = 1;
}

static int refresh_moduli(afd_mesh* m) {
  const Grid& g = m->gr;
  const size_t ne = g.nelem;
  k_convert<float><<<grid_blocks(ne, 256, 4096), 256, 0, m->s>>>(ne, m->E64, m->w32.E); m->launches++;
  const double d0 = elem_diag(m->opt.nu, m->opt.h);
  k_invdiag<float><<<grid_blocks(g.nnodes, 256, 4096), 256, 0, m->s>>>(g, m->E64, d0, m->w32.invdiag); m->launches++;
  k_expand3<float><<<grid_blocks(g.ndof, 256, 4096), 256, 0, m->s>>>(g.ndof, m->w32.invdiag, m->w32.invd); m->launches++;
  if (m->opt.precision == AFD_FP64) {   // the FP64 Jacobi factors serve only the FP64 solver
    k_invdiag<double><<<grid_blocks(g.nnodes, 256, 4096), 256, 0, m->s>>>(g, m->E64, d0, m->w64.invdiag); m->launches++;
    k_expand3<double><<<grid_blocks(g.ndof, 256, 4096), 256, 0, m->s>>>(g.ndof, m->w64.invdiag, m->w64.invd); m->launches++;
  }
  CK(cudaGetLastError());
  m->coarse_valid = false;
  m->has_moduli = true;
  return AFD_OK;
}

int afd_set_element_moduli(afd_mesh* m, const double* E, int on_device) {
  if (!m || !E) return fail(AFD_ERR_INVALID_ARG, "null argument");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  const size_t ne = m->gr.nelem;
  CK(cudaMemcpyAsync(m->E64, E, ne * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->s));
  int* bad = (int*)m->fsmall;
  CK(cudaMemsetAsync(bad, 0, sizeof(int), m->s));
  k_check_moduli<<<grid_blocks(ne, 256, 4096), 256, 0, m->s>>>(ne, m->E64, bad); m->launches++;
  int hbad = 0;
  CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, m->s));
  CK(cudaStreamSynchronize(m->s));
  if (hbad) {
    m->has_moduli = false;
    return fail(AFD_ERR_INVALID_ARG, "moduli must be finite and > 0");
  }
  TRY(refresh_moduli(m));
  return finish(m);
}

__global__ void k_pack_fixed(int nnodes, const uint8_t* __restrict__ dof_mask, uint8_t* __restrict__ node_bits) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nnodes; n += gridDim.x * blockDim.x)
    node_bits[n] = (dof_mask[3 * n] ? 1 : 0) | (dof_mask[3 * n + 1] ? 2 : 0) | (dof_mask[3 * n + 2] ? 4 : 0);
}

__global__ void k_zero_fixed(int nnodes, int nrhs, int vs, const uint8_t* __restrict__ bits, double* __restrict__ f) {
  const int rhs = blockIdx.y;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < nnodes; n += gridDim.x * blockDim.x) {
    const uint8_t b = bits[n];
    for (int c = 0; c < 3; ++c)
      if ((b >> c) & 1) f[(size_t)rhs * vs + 3 * n + c] = 0.0;
  }
}

static int reduce_partials_host(afd_mesh* m, int nrhs, int nparts, std::vector<double>& out) {
  std::vector<double> h((size_t)nrhs * nparts);
  CK(cudaMemcpyAsync(h.data(), m->partials, h.size() * sizeof(double), cudaMemcpyDeviceToHost, m->s));
  CK(cudaStreamSynchronize(m->s));
  out.assign(nrhs, 0.0);
  for (int r = 0; r < nrhs; ++r)
    for (int i = 0; i < nparts; ++i) out[r] += h[(size_t)r * nparts + i];
  return AFD_OK;
}

int afd_set_loads_bcs(afd_mesh* m, int n_rhs, const double* f, int f_on_device, const uint8_t* mask, int mask_on_device) {
  if (!m || !f || !mask) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (n_rhs < 1 || n_rhs > MAX_RHS) return fail(AFD_ERR_INVALID_ARG, "n_rhs must be in [1, %d]", MAX_RHS);
  DeviceGuard dg(m->device);
  TRY(enter(m));
  TRY(ensure_rhs(m, n_rhs));
  const Grid& g = m->gr;
  const size_t n = (size_t)n_rhs * g.vs;
  CK(cudaMemsetAsync(m->f64, 0, n * sizeof(double), m->s));
  CK(cudaMemcpy2DAsync(m->f64, (size_t)g.vs * sizeof(double), f, (size_t)g.ndof * sizeof(double),
                       (size_t)g.ndof * sizeof(double), n_rhs,
                       f_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->s));
  uint8_t* dmask = nullptr;
  if (mask_on_device) {
    dmask = (uint8_t*)mask;
  } else {
    TRY(dalloc(&dmask, (size_t)g.ndof));
    CK(cudaMemcpyAsync(dmask, mask, g.ndof, cudaMemcpyHostToDevice, m->s));
  }
  k_pack_fixed<<<grid_blocks(g.nnodes, 256, 4096), 256, 0, m->s>>>(g.nnodes, dmask, m->fixed); m->launches++;
  m->tflags_ty = 0;   // the packed-band stencil's tile flags follow the supports
  k_group_box_init<<<grid_blocks((size_t)6 * m->gp.ng, 256, 256), 256, 0, m->s>>>(m->gp.ng, m->gbox); m->launches++;
  k_group_fixed<<<grid_blocks(g.nnodes, 256, 4096), 256, 0, m->s>>>(g, m->gp, m->fixed, m->gbox); m->launches++;
  m->gbox_h.assign((size_t)6 * m->gp.ng, 0);
  CK(cudaMemcpyAsync(m->gbox_h.data(), m->gbox, (size_t)6 * m->gp.ng * sizeof(int), cudaMemcpyDeviceToHost, m->s));
  CK(cudaStreamSynchronize(m->s));
  {
    std::vector<long long> off(m->gp.ng + 1);
    size_t tot = 0;
    for (int G = 0; G < m->gp.ng; ++G) {
      off[G] = (long long)tot;
      tot += 18 * (size_t)node_shell_count(g, m->gp, G, m->gbox_h.data() + 6 * G);
    }
    off[m->gp.ng] = (long long)tot;
    if (tot > m->aw_total || !m->aw_node) {
      invalidate_graphs(m);
      dfree(m->aw_node);
      TRY(dalloc(&m->aw_node, tot / 18 + 1));
    }
    m->aw_total = tot;
    CK(cudaMemcpyAsync(m->aw_off, off.data(), (m->gp.ng + 1) * sizeof(long long), cudaMemcpyHostToDevice, m->s));
  }
  TRY(build_cut_records(m));
  k_zero_fixed<<<dim3(grid_blocks(g.nnodes, 256, 4096), n_rhs), 256, 0, m->s>>>(g.nnodes, n_rhs, g.vs, m->fixed, m->f64); m->launches++;
  CK(cudaMemsetAsync(m->u64, 0, n * sizeof(double), m->s));
  CK(cudaGetLastError());
  TRY(ensure_partials(m, (size_t)n_rhs * RED_BLOCKS));
  k_dot<double, double><<<dim3(RED_BLOCKS, n_rhs), RED_THREADS, 0, m->s>>>(g.ndof, g.vs, m->f64, m->f64, m->partials); m->launches++;
  std::vector<double> ff;
  TRY(reduce_partials_host(m, n_rhs, RED_BLOCKS, ff));
  if (!mask_on_device) cudaFree(dmask);
  m->fnorm.assign(n_rhs, 0.0);
  for (int r = 0; r < n_rhs; ++r) {
    if (!std::isfinite(ff[r])) return fail(AFD_ERR_INVALID_ARG, "load case %d is not finite", r);
    m->fnorm[r] = std::sqrt(ff[r]);
  }
  m->nrhs = n_rhs;
  m->has_loads = true;
  m->has_solution = false;
  m->coarse_valid = false;
  return finish(m);
}

// r = f - K u64 from FP64 data into its float copy b32 (nullable: the norm
// only); returns ||r||/||f|| per RHS.  dfl: the arithmetic is double-float
// (FP32 pairs, about 44 bits) instead of FP64.
static int true_residual(afd_mesh* m, float* b32, std::vector<double>& rel, bool dfl = false) {
  const int nsb = stencil_blocks(m, true);
  TRY(ensure_partials(m, (size_t)m->nrhs * std::max(nsb, 2 * RED_BLOCKS)));
  if (dfl)
    TRY((launch_stencil<double, ST_RESIDUAL, double, dfloat>(m, m->u64, nullptr, m->w64.E, m->f64, b32, m->partials,
                                                               nullptr, m->nrhs, m->w64.K)));
  else
    TRY((launch_stencil<double, ST_RESIDUAL, double>(m, m->u64, nullptr, m->w64.E, m->f64, b32, m->partials, nullptr,
                                                       m->nrhs, m->w64.K)));
  std::vector<double> rr;
  TRY(reduce_partials_host(m, m->nrhs, nsb, rr));
  if (dfl)
    for (int r = 0; r < m->nrhs; ++r)
      if (!std::isfinite(rr[r])) return true_residual(m, b32, rel, false);   // beyond FP32's exponent range
  rel.resize(m->nrhs);
  for (int r = 0; r < m->nrhs; ++r) rel[r] = m->fnorm[r] > 0 ? std::sqrt(rr[r]) / m->fnorm[r] : std::sqrt(rr[r]);
  return AFD_OK;
}

int afd_solve(afd_mesh* m, double rel_tol, int warm_start, afd_stats* per_rhs, double* u_out, int u_on_device) {
  if (!m) return fail(AFD_ERR_INVALID_ARG, "null mesh");
  if (!(rel_tol > 0.0) || !std::isfinite(rel_tol)) return fail(AFD_ERR_INVALID_ARG, "rel_tol must be > 0");
  if (!m->has_moduli || !m->has_loads) return fail(AFD_ERR_STATE, "set moduli and loads before solving");
  DeviceGuard dg(m->device);
  auto t0 = std::chrono::steady_clock::now();
  TRY(enter(m));
  const int R = m->nrhs;
  const Grid& g = m->gr;
  TRY(build_coarse(m));
  if (m->opt.autotune && !m->tuned && m->opt.precision == AFD_MIXED) {
    TRY(autotune_stencil(m));
    TRY(autotune_coarse_split(m));
  }
  const bool cold = !warm_start || !m->has_solution;
  if (cold) CK(cudaMemsetAsync(m->u64, 0, (size_t)R * g.vs * sizeof(double), m->s));
  std::vector<int> iters(R, 0), status(R, AFD_OK), refine(R, 0);
  std::vector<double> rel;
  if (m->opt.precision == AFD_FP64) {
    TRY(ensure_work(m, m->w64, R));
    std::vector<double> t2(R);
    std::vector<int> act(R, 1);
      // the recursive residual drifts from the true one: aim 10% below the tolerance
    for (int r = 0; r < R; ++r) t2[r] = (0.9 * rel_tol * m->fnorm[r]) * (0.9 * rel_tol * m->fnorm[r]);
    std::vector<CGState> st;
    TRY((dpcg<double, double>(m, m->w64, m->f64, m->u64, cold, R, t2, act, m->opt.max_iter, st)));
    for (int r = 0; r < R; ++r) {
      iters[r] = st[r].iters;
      status[r] = st[r].status;
    }
    TRY(true_residual(m, nullptr, rel));
  } else {
    TRY(ensure_work(m, m->w32, R));
    float* b32 = m->w32.b;
    // the refinement residual in double-float unless the tolerance nears its rounding (about 1e-12 of
    // ||f||) or the loads are far from unit scale (the pairs have FP32's exponent range)
    bool dfl = !m->opt.residual_fp64 && rel_tol >= RESIDUAL_DF_MIN_TOL;
    for (int r = 0; r < R; ++r)
      if (m->fnorm[r] != 0.0 && !(m->fnorm[r] >= 1e-20 && m->fnorm[r] <= 1e20)) dfl = false;
    if (cold) {
      // u = 0: the residual is f itself (zero on fixed DOFs), so the first FP64 pass is not needed
      for (int r = 0; r < R; ++r) {
        k_convert<float><<<grid_blocks(g.ndof, 256, 4096), 256, 0, m->s>>>((size_t)g.ndof, m->f64 + (size_t)r * g.vs,
                                                                          b32 + (size_t)r * g.vs);
        m->launches++;
      }
      CK(cudaGetLastError());
      rel.assign(R, 0.0);
      for (int r = 0; r < R; ++r) rel[r] = m->fnorm[r] > 0.0 ? 1.0 : 0.0;
    } else {
      TRY(true_residual(m, b32, rel, dfl));
    }
    for (int step = 0; step <= m->opt.max_refine; ++step) {
      std::vector<int> act(R, 0);
      std::vector<double> t2(R, 0.0);
      bool any = false;
      for (int r = 0; r < R; ++r) {
        if (!std::isfinite(rel[r])) { status[r] = AFD_ERR_NAN; continue; }
        if (rel[r] <= rel_tol || m->fnorm[r] == 0.0) continue;
        if (step == m->opt.max_refine || iters[r] >= m->opt.max_iter) { status[r] = AFD_ERR_NOT_CONVERGED; continue; }
        act[r] = 1;
        any = true;
        double eta = std::min(0.5, std::max(m->opt.inner_tol, m->opt.inner_aim * rel_tol / rel[r]));
        const double rn = rel[r] * (m->fnorm[r] > 0 ? m->fnorm[r] : 1.0);
        t2[r] = (eta * rn) * (eta * rn);
      }
      if (!any) break;
      CK(cudaMemsetAsync(m->w32.x, 0, (size_t)R * g.vs * sizeof(float), m->s));
      std::vector<CGState> st;
      int budget = m->opt.max_iter;
      for (int r = 0; r < R; ++r) if (act[r]) budget = std::min(budget, std::max(1, m->opt.max_iter - iters[r]));
      TRY((dpcg<float, float>(m, m->w32, b32, m->w32.x, true, R, t2, act, budget, st)));
      std::vector<int> skip(R);
      for (int r = 0; r < R; ++r) {
        skip[r] = !act[r];
        if (act[r]) {
          iters[r] += st[r].iters;
          refine[r] += 1;
          if (st[r].status == AFD_ERR_NAN) status[r] = AFD_ERR_NAN;
        }
      }
      int* dskip = m->done;
      CK(cudaMemcpyAsync(dskip, skip.data(), R * sizeof(int), cudaMemcpyHostToDevice, m->s));
      k_accumulate<<<dim3(grid_blocks(g.ndof, 256, 2048), R), 256, 0, m->s>>>(g.ndof, g.vs, m->u64, m->w32.x, dskip); m->launches++;
      CK(cudaGetLastError());
      TRY(true_residual(m, b32, rel, dfl));
    }
    for (int r = 0; r < R; ++r)
      if (status[r] == AFD_OK && !(rel[r] <= rel_tol)) status[r] = AFD_ERR_NOT_CONVERGED;
  }
  m->has_solution = true;
  if (u_out)
    CK(cudaMemcpy2DAsync(u_out, (size_t)g.ndof * sizeof(double), m->u64, (size_t)g.vs * sizeof(double),
                         (size_t)g.ndof * sizeof(double), R,
                         u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->s));
  TRY(finish(m));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int rc = AFD_OK;
  for (int r = 0; r < R; ++r) {
    if (m->opt.precision == AFD_FP64 && status[r] == AFD_OK && !(rel[r] <= rel_tol * 1.0000001)) status[r] = AFD_ERR_NOT_CONVERGED;
    if (status[r] != AFD_OK && rc == AFD_OK) rc = status[r];
    if (per_rhs) {
      per_rhs[r].iters = iters[r];
      per_rhs[r].refine_steps = refine[r];
      per_rhs[r].rel_residual = rel[r];
      per_rhs[r].ms = ms;
      per_rhs[r].status = status[r];
    }
  }
  if (rc != AFD_OK) fail(rc, "solve did not reach rel_tol %.3g for every load case", rel_tol);
  return rc;
}

int afd_compliance(afd_mesh* m, double* J_out) {
  if (!m || !J_out) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (!m->has_solution) return fail(AFD_ERR_STATE, "no solution");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  TRY(ensure_partials(m, (size_t)m->nrhs * RED_BLOCKS));
  k_dot<double, double><<<dim3(RED_BLOCKS, m->nrhs), RED_THREADS, 0, m->s>>>(m->gr.ndof, m->gr.vs, m->f64, m->u64, m->partials); m->launches++;
  CK(cudaGetLastError());
  std::vector<double> J;
  TRY(reduce_partials_host(m, m->nrhs, RED_BLOCKS, J));
  for (int r = 0; r < m->nrhs; ++r) J_out[r] = J[r];
  return finish(m);
}

static int fields_to(afd_mesh* m, int kind, float* out) {
  FieldConsts F;
  const double nu = m->opt.nu;
  F.lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  F.mu = 1.0 / (2.0 * (1.0 + nu));
  F.nu = nu;
  F.inv4h = 1.0 / (4.0 * m->opt.h);
  const dim3 grid(grid_blocks(m->gr.nelem, 256, 8 * RED_BLOCKS), m->nrhs);
  if (m->opt.precision == AFD_FP64) {
    k_element_fields<double><<<grid, 256, 0, m->s>>>(m->gr, m->u64, m->E64, m->w64.K, F, kind, out); m->launches++;
  } else {
    k_element_fields<float><<<grid, 256, 0, m->s>>>(m->gr, m->u64, m->E64, m->w32.K, F, kind, out); m->launches++;
  }
  CK(cudaGetLastError());
  return AFD_OK;
}

int afd_sensitivity(afd_mesh* m, int kind, float* out, int out_on_device) {
  if (!m || !out) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (kind < 0 || kind > 2) return fail(AFD_ERR_INVALID_ARG, "unknown sensitivity kind %d", kind);
  if (!m->has_solution) return fail(AFD_ERR_STATE, "no solution");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  TRY(fields_to(m, kind, m->fbuf));
  CK(cudaMemcpyAsync(out, m->fbuf, (size_t)m->nrhs * m->gr.nelem * sizeof(float),
                     out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->s));
  TRY(finish(m));
  m->fcache_kind = kind;
  return AFD_OK;
}

static int maxabs_per_rhs(afd_mesh* m, const float* x, int nrhs, float* dmax_out) {
  float* part = m->fsmall + FS_PARTS;
  const int nb = std::min(FS_MAX_BLOCKS, grid_blocks(m->gr.nelem));
  k_maxabs_partial<<<dim3(nb, nrhs), 256, 0, m->s>>>(m->gr.nelem, x, part); m->launches++;
  k_max_finalize<<<nrhs, 256, 0, m->s>>>(nb, part, dmax_out); m->launches++;
  CK(cudaGetLastError());
  return AFD_OK;
}

int afd_pnorm_stress(afd_mesh* m, double p, double* out) {
  if (!m || !out) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (!(p >= 1.0) || !std::isfinite(p)) return fail(AFD_ERR_INVALID_ARG, "p must be >= 1");
  if (!m->has_solution) return fail(AFD_ERR_STATE, "no solution");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  const int R = m->nrhs;
  TRY(fields_to(m, AFD_SENS_VON_MISES, m->fbuf));
  float* dmaxv = m->fsmall + FS_MAXV;
  TRY(maxabs_per_rhs(m, m->fbuf, R, dmaxv));
  TRY(ensure_partials(m, (size_t)R * RED_BLOCKS));
  k_pow_partial<<<dim3(RED_BLOCKS, R), 256, 0, m->s>>>(m->gr.nelem, m->fbuf, dmaxv, p, m->partials); m->launches++;
  CK(cudaGetLastError());
  std::vector<double> s;
  TRY(reduce_partials_host(m, R, RED_BLOCKS, s));
  std::vector<float> mx(R);
  CK(cudaMemcpyAsync(mx.data(), dmaxv, R * sizeof(float), cudaMemcpyDeviceToHost, m->s));
  CK(cudaStreamSynchronize(m->s));
  for (int r = 0; r < R; ++r) out[r] = (double)mx[r] * std::pow(s[r], 1.0 / p);
  return finish(m);
}

int afd_stress_sensitivity(afd_mesh* m, double p, double rel_tol, float* out, int out_on_device, afd_stats* adj_stats,
                           double* lambda_out, int lambda_on_device) {
  if (!m || !out) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (!(p >= 1.0) || !std::isfinite(p)) return fail(AFD_ERR_INVALID_ARG, "p must be >= 1");
  if (!(rel_tol > 0.0) || !std::isfinite(rel_tol)) return fail(AFD_ERR_INVALID_ARG, "rel_tol must be > 0");
  if (!m->has_solution) return fail(AFD_ERR_STATE, "no solution");
  const int R = m->nrhs;
  std::vector<double> pn(R);
  TRY(afd_pnorm_stress(m, p, pn.data()));
  DeviceGuard dg(m->device);
  TRY(enter(m));
  const Grid& g = m->gr;
  if (m->adj_cap < R) {
    dfree(m->lam64); dfree(m->gadj); dfree(m->dsig); dfree(m->pn_d);
    m->adj_cap = 0;
    TRY(dalloc(&m->lam64, (size_t)R * g.vs));
    TRY(dalloc(&m->gadj, (size_t)R * g.vs));
    TRY(dalloc(&m->dsig, (size_t)R * 6 * g.nelem));
    TRY(dalloc(&m->pn_d, (size_t)R));
    m->adj_cap = R;
  }
  FieldConsts F;
  const double nu = m->opt.nu;
  F.lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  F.mu = 1.0 / (2.0 * (1.0 + nu));
  F.nu = nu;
  F.inv4h = 1.0 / (4.0 * m->opt.h);
  CK(cudaMemcpyAsync(m->pn_d, pn.data(), R * sizeof(double), cudaMemcpyHostToDevice, m->s));
  k_pnorm_dsig<<<dim3(grid_blocks(g.nelem, 256, 8 * RED_BLOCKS), R), 256, 0, m->s>>>(g, m->u64, m->E64, F, p, m->pn_d,
                                                                                    m->dsig); m->launches++;
  CK(cudaMemsetAsync(m->gadj, 0, (size_t)R * g.vs * sizeof(double), m->s));
  k_pnorm_adjoint_rhs<<<dim3(grid_blocks(g.nnodes, 256, 8 * RED_BLOCKS), R), 256, 0, m->s>>>(g, m->dsig, m->fixed,
                                                                                            F.inv4h, m->gadj); m->launches++;
  TRY(ensure_partials(m, (size_t)R * RED_BLOCKS));
  k_dot<double, double><<<dim3(RED_BLOCKS, R), RED_THREADS, 0, m->s>>>(g.ndof, g.vs, m->gadj, m->gadj, m->partials); m->launches++;
  CK(cudaGetLastError());
  std::vector<double> gg;
  TRY(reduce_partials_host(m, R, RED_BLOCKS, gg));
  std::vector<double> gnorm(R);
  for (int r = 0; r < R; ++r) gnorm[r] = std::sqrt(gg[r]);
  // the adjoint problem K lambda = g on the same mesh, moduli, supports and coarse space:
  // swap it into the load / solution buffers for one solve, then swap back
  std::swap(m->f64, m->gadj);
  std::swap(m->u64, m->lam64);
  std::swap(m->fnorm, gnorm);
  invalidate_graphs(m);
  const int rc = afd_solve(m, rel_tol, 0, adj_stats, nullptr, 0);
  const std::string err = g_err;
  std::swap(m->f64, m->gadj);
  std::swap(m->u64, m->lam64);
  std::swap(m->fnorm, gnorm);
  invalidate_graphs(m);
  m->has_solution = true;
  if (rc != AFD_OK && rc != AFD_ERR_NOT_CONVERGED) return fail(rc, "adjoint solve: %s", err.c_str());
  float* dst = out_on_device ? out : m->fbuf;
  k_stress_topo<<<dim3(grid_blocks(g.nelem, 256, 8 * RED_BLOCKS), R), 256, 0, m->s>>>(g, m->u64, m->lam64, m->E64, F,
                                                                                      dst); m->launches++;
  CK(cudaGetLastError());
  if (!out_on_device)
    CK(cudaMemcpyAsync(out, m->fbuf, (size_t)R * g.nelem * sizeof(float), cudaMemcpyDeviceToHost, m->s));
  if (lambda_out)
    CK(cudaMemcpy2DAsync(lambda_out, (size_t)g.ndof * sizeof(double), m->lam64, (size_t)g.vs * sizeof(double),
                         (size_t)g.ndof * sizeof(double), R,
                         lambda_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->s));
  TRY(finish(m));
  if (rc != AFD_OK) return fail(rc, "adjoint solve did not reach rel_tol %.3g", rel_tol);
  return AFD_OK;
}

// ---------------------------------------------------------------------------
// Modal analysis (the eigenvalue constraint of Sec. 3.8; Eq. 3.4 needs its
// modes) and linear buckling (Eq. 3.5): block LOBPCG on the mesh's own solver.
// ---------------------------------------------------------------------------
constexpr int MODAL_GRAM_BLOCKS = 304;

static int modal_gram(afd_mesh* m, int kp, const double* Y, const double* Z, double* out) {
  const Grid& g = m->gr;
  k_gram<<<MODAL_GRAM_BLOCKS, 256, 0, m->s>>>(g.ndof, g.vs, kp, Y, Z, m->mparts); m->launches++;
  k_gram_final<<<1, 256, 0, m->s>>>(MODAL_GRAM_BLOCKS, kp * kp, m->mparts, out); m->launches++;
  CK(cudaGetLastError());
  return AFD_OK;
}

// The geometric element table c_geo[q][a][b] for the unit cube: the integrals
// of d_k N_a d_l N_b, in closed form per axis (1D integrals of the linear
// shape functions: int phi_p phi_q = 1/3 or 1/6, int phi_p' phi_q = (2p - 1)/2,
// int phi_p' phi_q' = (2p - 1)(2q - 1)), summed over (k, l) and (l, k) for the
// off-diagonal stress components q = xy, yz, zx.  A cube of edge h scales
// them by h, which the state stress carries (k_state_stress), so the table is
// the same for every mesh and concurrent uploads cannot disagree.
static int upload_geo_table(afd_mesh* m) {
  const double h = 1.0;
  static const int kk[6] = {0, 1, 2, 0, 1, 2}, ll[6] = {0, 1, 2, 1, 2, 0};
  double t[6][8][8];
  auto bit = [](int a, int d) { return (a >> d) & 1; };
  auto m1 = [](int p, int q) { return p == q ? 1.0 / 3.0 : 1.0 / 6.0; };
  auto H = [&](int k, int l, int a, int b) {
    if (k == l) {
      double v = h * (2 * bit(a, k) - 1) * (2 * bit(b, k) - 1);
      for (int d = 0; d < 3; ++d)
        if (d != k) v *= m1(bit(a, d), bit(b, d));
      return v;
    }
    const int mm = 3 - k - l;
    return h * 0.5 * (2 * bit(a, k) - 1) * 0.5 * (2 * bit(b, l) - 1) * m1(bit(a, mm), bit(b, mm));
  };
  for (int q = 0; q < 6; ++q)
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b)
        t[q][a][b] = q < 3 ? H(kk[q], kk[q], a, b) : H(kk[q], ll[q], a, b) + H(ll[q], kk[q], a, b);
  CK(cudaMemcpyToSymbolAsync(c_geo, t, sizeof(t), 0, cudaMemcpyHostToDevice, m->s));
  return AFD_OK;
}

// Block LOBPCG for the kp smallest theta of A phi = theta B phi on the free
// DOFs, preconditioned by K^-1 (the mesh's solver, relative tolerance
// EIG_PREC_TOL), with soft locking of converged vectors.
//   EIG_MODAL:    A = K, B = M (lumped mass in mmass), theta = lambda.
//   EIG_BUCKLING: A = K_G, B = K, theta = -1/lambda, so the most negative
//                 theta is the smallest positive load factor.  (Subspace
//                 iteration would follow the largest |theta|, and under many
//                 loads the reversed load's factors, theta > 0, are larger.)
// Each step: the residual block R = A X - B X Theta, W = K^-1 R, the images
// A W and B W, then Rayleigh-Ritz on span[X, W, P] (rows contiguous in lS,
// images in lAS / lBS) with FP64 Gram matrices and the truncating small
// eigensolver; X and the new direction P (the W, P part of the Ritz
// coefficients) are rebuilt with their images into the other buffer.
// Converged when |R_r| <= tol |theta_r| |B X_r| for the first n_modes.
// vals: the kp Ritz values theta; the B-normalised Ritz vectors end in mX.
enum EigKind { EIG_MODAL = 0, EIG_BUCKLING = 1 };
// Relative tolerance of the preconditioner solves.  On the voided 128x64x64
// cantilever, 1e-3 / 1e-2 / 3e-2 / 1e-1 took 881 / 726 / 556 / 446 inner
// iterations for 4 modes (8 / 9 / 9 / 10 steps) and 2908 / 1870 / 1310 / 987
// for 2 buckling factors (40 / 42 / 44 / 53 steps); 3e-2 was the fastest for
// both (the steps' own cost grows with their number).
constexpr double EIG_PREC_TOL = 3e-2;
static int lobpcg(afd_mesh* m, EigKind kind, int n_modes, int kp, double tol, int max_iter, std::vector<double>& vals,
                  bool& converged, int& steps, int& solve_iters) {
  const Grid& g = m->gr;
  const size_t blk = (size_t)kp * g.vs;
  const dim3 vgrid(grid_blocks(g.ndof, 256, 2048), kp);
  const dim3 ngrid(grid_blocks(g.nnodes, 256, 2048), kp);
  const unsigned cb = grid_blocks(g.ndof, 256, 2048);
  int cur = 0;
  steps = solve_iters = 0;
  converged = false;
  vals.assign(kp, 0.0);
  std::vector<double> V;
  auto images = [&](const double* Xs, double* AXs, double* BXs) -> int {   // A and B of kp rows
    double* KXs = kind == EIG_MODAL ? AXs : BXs;
    // K X from the FP64 block: in double-float arithmetic on mixed meshes (a few 2^-44 of the element forces,
    // on the FP32 pipes), in FP64 on FP64 meshes
    if (m->opt.precision == AFD_MIXED)
      TRY((launch_stencil<double, ST_APPLY, double, dfloat>(m, Xs, KXs, m->w64.E, nullptr, nullptr, nullptr, nullptr,
                                                              kp, m->w64.K)));
    else
      TRY((launch_stencil<double, ST_APPLY, double>(m, Xs, KXs, m->w64.E, nullptr, nullptr, nullptr, nullptr, kp,
                                                      m->w64.K)));
    if (kind == EIG_MODAL) {
      k_mass_apply<<<vgrid, 256, 0, m->s>>>(g.ndof, g.vs, m->mmass, Xs, BXs); m->launches++;
    } else {
      k_geo_apply<<<ngrid, 256, 0, m->s>>>(g, m->bS6, m->fixed, 1.0, Xs, AXs); m->launches++;
    }
    CK(cudaGetLastError());
    return AFD_OK;
  };
  auto rayleigh_ritz = [&](int mrows, std::vector<double>& th, std::vector<double>& Vh) -> int {
    TRY(modal_gram(m, mrows, m->lS[cur], m->lAS[cur], m->mA));
    TRY(modal_gram(m, mrows, m->lS[cur], m->lBS[cur], m->mB));
    k_small_geig_robust<<<1, 32, 0, m->s>>>(mrows, kp, m->mA, m->mB, m->mlam, m->mV, m->minfo); m->launches++;
    int info = 0;
    th.assign(kp, 0.0);
    Vh.assign((size_t)mrows * kp, 0.0);
    CK(cudaMemcpyAsync(th.data(), m->mlam, kp * sizeof(double), cudaMemcpyDeviceToHost, m->s));
    CK(cudaMemcpyAsync(Vh.data(), m->mV, Vh.size() * sizeof(double), cudaMemcpyDeviceToHost, m->s));
    CK(cudaMemcpyAsync(&info, m->minfo, sizeof(int), cudaMemcpyDeviceToHost, m->s));
    CK(cudaStreamSynchronize(m->s));
    if (info != 0)
      return fail(AFD_ERR_NAN, "Rayleigh-Ritz step failed (%s)",
                  info == 3 ? "the block lost rank" : "Jacobi sweeps did not converge");
    for (double t : th)
      if (!std::isfinite(t)) return fail(AFD_ERR_NAN, "eigen iteration is not finite");
    return AFD_OK;
  };
  // X and P (with_p) of the next buffer from the coefficients of span[X, W, P]
  auto rebuild = [&](int mrows, const std::vector<double>& Vh, bool with_p) -> int {
    const int nxt = 1 - cur;
    const double* src[3] = {m->lS[cur], m->lAS[cur], m->lBS[cur]};
    double* dst[3] = {m->lS[nxt], m->lAS[nxt], m->lBS[nxt]};
    CK(cudaMemcpyAsync(m->mV, Vh.data(), Vh.size() * sizeof(double), cudaMemcpyHostToDevice, m->s));
    for (int q = 0; q < 3; ++q) {
      k_block_combine<<<cb, 256, 0, m->s>>>(g.ndof, g.vs, mrows, kp, src[q], m->mV, dst[q]); m->launches++;
    }
    if (with_p) {
      std::vector<double> Vp(Vh);
      for (int i = 0; i < kp; ++i)
        for (int c = 0; c < kp; ++c) Vp[(size_t)i * kp + c] = 0.0;   // drop the X rows: P = W Vw + P Vp
      CK(cudaMemcpyAsync(m->mB, Vp.data(), Vp.size() * sizeof(double), cudaMemcpyHostToDevice, m->s));
      for (int q = 0; q < 3; ++q) {
        k_block_combine<<<cb, 256, 0, m->s>>>(g.ndof, g.vs, mrows, kp, src[q], m->mB, dst[q] + 2 * blk);
        m->launches++;
      }
    }
    CK(cudaGetLastError());
    cur = nxt;
    return AFD_OK;
  };
  // start: random X, Rayleigh-Ritz on X alone
  k_modal_start<<<vgrid, 256, 0, m->s>>>(g.ndof, g.vs, 0x2203151150ull, m->mmass, m->lS[cur]); m->launches++;
  TRY(images(m->lS[cur], m->lAS[cur], m->lBS[cur]));
  TRY(rayleigh_ritz(kp, vals, V));
  TRY(rebuild(kp, V, false));
  bool have_p = false;
  TRY(ensure_partials(m, (size_t)kp * 2 * RED_BLOCKS));
  for (int it = 0; it < max_iter; ++it) {
    // residual block into the solver's load buffer, its norms, the convergence test
    CK(cudaMemcpyAsync(m->bcoef, vals.data(), kp * sizeof(double), cudaMemcpyHostToDevice, m->s));
    TRY(ensure_partials(m, (size_t)kp * 2 * RED_BLOCKS));
    k_lobpcg_residual<<<dim3(RED_BLOCKS, kp), RED_THREADS, 0, m->s>>>(g.ndof, g.vs, m->lAS[cur], m->lBS[cur],
                                                                     m->mmass, m->bcoef, m->f64, m->partials);
    m->launches++;
    CK(cudaGetLastError());
    std::vector<double> hp((size_t)kp * RED_BLOCKS * 2);
    CK(cudaMemcpyAsync(hp.data(), m->partials, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, m->s));
    CK(cudaStreamSynchronize(m->s));
    std::vector<double> rn(kp, 0.0), kn(kp, 0.0);
    for (int r = 0; r < kp; ++r)
      for (int b = 0; b < RED_BLOCKS; ++b) {
        rn[r] += hp[((size_t)r * RED_BLOCKS + b) * 2];
        kn[r] += hp[((size_t)r * RED_BLOCKS + b) * 2 + 1];
      }
    std::vector<int> locked(kp, 0);
    for (int r = 0; r < kp; ++r) locked[r] = std::sqrt(rn[r]) <= tol * std::fabs(vals[r]) * std::sqrt(kn[r]);
    converged = true;
    for (int r = 0; r < n_modes; ++r)
      if (!locked[r]) converged = false;
    if (converged) break;
    // W = K^-1 R.  Soft locking: a vector that already meets the test adds no
    // direction (its residual column is zeroed, so the solver skips it and the
    // Rayleigh-Ritz step drops the zero column); directions of converged
    // vectors are mostly noise and make the basis dependent.
    m->nrhs = kp;
    m->fnorm.assign(kp, 0.0);
    for (int r = 0; r < kp; ++r) {
      m->fnorm[r] = locked[r] ? 0.0 : std::sqrt(rn[r]);
      if (locked[r]) CK(cudaMemsetAsync(m->f64 + (size_t)r * g.vs, 0, (size_t)g.ndof * sizeof(double), m->s));
    }
    std::vector<afd_stats> st(kp);
    const int src = afd_solve(m, EIG_PREC_TOL, 0, st.data(), nullptr, 0);
    if (src != AFD_OK && src != AFD_ERR_NOT_CONVERGED) return src;
    int mx = 0;
    for (int r = 0; r < kp; ++r) mx = std::max(mx, st[r].iters);
    solve_iters += mx;
    CK(cudaMemcpyAsync(m->lS[cur] + blk, m->u64, blk * sizeof(double), cudaMemcpyDeviceToDevice, m->s));
    TRY(images(m->lS[cur] + blk, m->lAS[cur] + blk, m->lBS[cur] + blk));
    const int mrows = have_p ? 3 * kp : 2 * kp;
    TRY(rayleigh_ritz(mrows, vals, V));
    TRY(rebuild(mrows, V, true));
    have_p = true;
    steps = it + 1;
  }
  // the modes in mX for the sensitivity and the caller
  CK(cudaMemcpyAsync(m->mX, m->lS[cur], blk * sizeof(double), cudaMemcpyDeviceToDevice, m->s));
  return AFD_OK;
}

// Buffers of the eigensolvers for a block of kp vectors: the modes, the mass
// (or free-DOF mask), the small matrices, the LOBPCG blocks [X, W, P] with
// their A and B images (two of each), and for buckling the state stress and
// the load factors.
static int ensure_eig_buffers(afd_mesh* m, int kp, bool buckling) {
  const Grid& g = m->gr;
  if (m->modal_cap < kp) {
    dfree(m->mX); dfree(m->mmass); dfree(m->mparts);
    dfree(m->mA); dfree(m->mB); dfree(m->mV); dfree(m->mlam); dfree(m->minfo);
    m->modal_cap = 0;
    TRY(dalloc(&m->mX, (size_t)kp * g.vs));
    TRY(dalloc(&m->mmass, (size_t)g.vs));
    TRY(dalloc(&m->mparts, (size_t)MODAL_GRAM_BLOCKS * MODAL_MAX * MODAL_MAX));
    TRY(dalloc(&m->mA, (size_t)MODAL_MAX * MODAL_MAX));
    TRY(dalloc(&m->mB, (size_t)MODAL_MAX * MODAL_MAX));
    TRY(dalloc(&m->mV, (size_t)MODAL_MAX * MODAL_MAX));
    TRY(dalloc(&m->mlam, (size_t)MODAL_MAX));
    TRY(dalloc(&m->minfo, 1));
    m->modal_cap = kp;
  }
  if (!m->bcoef) TRY(dalloc(&m->bcoef, (size_t)MODAL_MAX));
  if (buckling && !m->bS6) TRY(dalloc(&m->bS6, (size_t)6 * g.nelem));
  {
    if (m->lobpcg_cap < kp) {
      for (int q = 0; q < 2; ++q) {
        dfree(m->lS[q]); dfree(m->lBS[q]); dfree(m->lAS[q]);
        TRY(dalloc(&m->lS[q], (size_t)3 * kp * g.vs));
        TRY(dalloc(&m->lBS[q], (size_t)3 * kp * g.vs));
        TRY(dalloc(&m->lAS[q], (size_t)3 * kp * g.vs));
      }
      m->lobpcg_cap = kp;
    }
  }
  return AFD_OK;
}

// Saves the load cases, runs `body`, restores them; the static solution is discarded.
template <typename F>
static int with_saved_loads(afd_mesh* m, F&& body) {
  const Grid& g = m->gr;
  const int R0 = m->nrhs;
  const std::vector<double> fnorm0 = m->fnorm;
  double* fsave = nullptr;
  TRY(dalloc(&fsave, (size_t)R0 * g.vs));
  CK(cudaMemcpyAsync(fsave, m->f64, (size_t)R0 * g.vs * sizeof(double), cudaMemcpyDeviceToDevice, m->s));
  const int rc = body();
  const std::string err = g_err;
  if (m->f64 && m->cap >= R0)
    CK(cudaMemcpyAsync(m->f64, fsave, (size_t)R0 * g.vs * sizeof(double), cudaMemcpyDeviceToDevice, m->s));
  CK(cudaStreamSynchronize(m->s));
  dfree(fsave);
  m->nrhs = R0;
  m->fnorm = fnorm0;
  m->has_solution = false;
  invalidate_graphs(m);
  TRY(finish(m));
  if (rc != AFD_OK) g_err = err;
  return rc;
}

// The LOBPCG block: the requested modes and two guard vectors; the
// Rayleigh-Ritz basis [X, W, P] holds 3 kp <= MODAL_MAX vectors.
constexpr int EIG_MAX_MODES = MODAL_MAX / 3 - 2;
static int eig_block(int n_modes, int& kp) {
  kp = n_modes + 2;
  if (n_modes < 1 || n_modes > EIG_MAX_MODES)
    return fail(AFD_ERR_INVALID_ARG, "n_modes must be in [1, %d]", EIG_MAX_MODES);
  return AFD_OK;
}

int afd_modal(afd_mesh* m, int n_modes, double rho, double tol, int max_iter, double* lam_out, double* modes_out,
              int modes_on_device, int* iters_out, int* solve_iters_out) {
  if (!m || !lam_out) return fail(AFD_ERR_INVALID_ARG, "null argument");
  int kp = 0;
  TRY(eig_block(n_modes, kp));
  if (!(rho > 0.0) || !std::isfinite(rho)) return fail(AFD_ERR_INVALID_ARG, "rho must be > 0");
  if (!(tol > 0.0) || !std::isfinite(tol) || max_iter < 1) return fail(AFD_ERR_INVALID_ARG, "bad tol / max_iter");
  if (!m->has_moduli || !m->has_loads) return fail(AFD_ERR_STATE, "set moduli and supports before afd_modal");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  const Grid& g = m->gr;
  bool converged = false;
  const int rc = with_saved_loads(m, [&]() -> int {
    TRY(ensure_rhs(m, kp));
    TRY(ensure_eig_buffers(m, kp, false));
    m->modal_valid = false;
    m->buckling_valid = false;
    const double h = m->opt.h;
    CK(cudaMemsetAsync(m->mmass, 0, (size_t)g.vs * sizeof(double), m->s));
    CK(cudaMemsetAsync(m->mX, 0, (size_t)kp * g.vs * sizeof(double), m->s));
    k_lumped_mass<<<grid_blocks(g.nnodes, 256, 4096), 256, 0, m->s>>>(g, m->E64, rho * h * h * h / 8.0, m->fixed,
                                                                      m->mmass); m->launches++;
    std::vector<double> vals;
    int steps = 0, solve_iters = 0;
    TRY(lobpcg(m, EIG_MODAL, n_modes, kp, tol, max_iter, vals, converged, steps, solve_iters));
    for (int r = 0; r < n_modes; ++r)
      if (!(vals[r] > 0.0)) return fail(AFD_ERR_NAN, "a non-positive eigenvalue: the supports leave a rigid mode");
    for (int r = 0; r < n_modes; ++r) lam_out[r] = vals[r];
    if (modes_out)
      CK(cudaMemcpy2DAsync(modes_out, (size_t)g.ndof * sizeof(double), m->mX, (size_t)g.vs * sizeof(double),
                           (size_t)g.ndof * sizeof(double), n_modes,
                           modes_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->s));
    if (iters_out) *iters_out = steps;
    if (solve_iters_out) *solve_iters_out = solve_iters;
    m->modal_n = n_modes;
    m->modal_rho = rho;
    m->modal_valid = true;
    return AFD_OK;
  });
  if (rc != AFD_OK) return fail(rc, "%s", g_err.c_str());
  if (!converged) return fail(AFD_ERR_NOT_CONVERGED, "modal iteration did not reach tol %.3g in %d steps", tol, max_iter);
  return AFD_OK;
}

int afd_buckling(afd_mesh* m, int n_modes, double tol, int max_iter, double* lam_out, double* modes_out,
                 int modes_on_device, int* iters_out, int* solve_iters_out) {
  if (!m || !lam_out) return fail(AFD_ERR_INVALID_ARG, "null argument");
  int kp = 0;
  TRY(eig_block(n_modes, kp));
  if (!(tol > 0.0) || !std::isfinite(tol) || max_iter < 1) return fail(AFD_ERR_INVALID_ARG, "bad tol / max_iter");
  if (!m->has_solution) return fail(AFD_ERR_STATE, "no static solution: afd_solve first (load case 0 is the state)");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  const Grid& g = m->gr;
  bool converged = false;
  // the state stress of load case 0 before anything overwrites the solution
  TRY(ensure_eig_buffers(m, kp, true));
  FieldConsts F;
  const double nu = m->opt.nu;
  F.lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  F.mu = 1.0 / (2.0 * (1.0 + nu));
  F.nu = nu;
  F.inv4h = 1.0 / (4.0 * m->opt.h);
  k_state_stress<<<grid_blocks(g.nelem, 256, 8 * RED_BLOCKS), 256, 0, m->s>>>(g, m->u64, m->E64, F, m->opt.h,
                                                                              m->bS6);
  m->launches++;
  TRY(upload_geo_table(m));
  const int rc = with_saved_loads(m, [&]() -> int {
    TRY(ensure_rhs(m, kp));
    TRY(ensure_eig_buffers(m, kp, true));
    m->modal_valid = false;
    m->buckling_valid = false;
    // the free-DOF mask of the residual (any positive value on free DOFs)
    CK(cudaMemsetAsync(m->mmass, 0, (size_t)g.vs * sizeof(double), m->s));
    CK(cudaMemsetAsync(m->mX, 0, (size_t)kp * g.vs * sizeof(double), m->s));
    k_lumped_mass<<<grid_blocks(g.nnodes, 256, 4096), 256, 0, m->s>>>(g, m->E64, 1.0, m->fixed, m->mmass);
    m->launches++;
    std::vector<double> vals;
    int steps = 0, solve_iters = 0;
    TRY(lobpcg(m, EIG_BUCKLING, n_modes, kp, tol, max_iter, vals, converged, steps, solve_iters));
    for (int r = 0; r < n_modes; ++r)
      if (!(vals[r] < 0.0)) return fail(AFD_ERR_NAN, "fewer than %d positive buckling factors for this load", n_modes);
    std::vector<double> lam(n_modes);
    for (int r = 0; r < n_modes; ++r) lam[r] = lam_out[r] = -1.0 / vals[r];
    CK(cudaMemcpyAsync(m->bcoef, lam.data(), n_modes * sizeof(double), cudaMemcpyHostToDevice, m->s));
    if (modes_out)
      CK(cudaMemcpy2DAsync(modes_out, (size_t)g.ndof * sizeof(double), m->mX, (size_t)g.vs * sizeof(double),
                           (size_t)g.ndof * sizeof(double), n_modes,
                           modes_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->s));
    if (iters_out) *iters_out = steps;
    if (solve_iters_out) *solve_iters_out = solve_iters;
    m->modal_n = n_modes;
    m->buckling_valid = true;
    return AFD_OK;
  });
  if (rc != AFD_OK) return fail(rc, "%s", g_err.c_str());
  if (!converged)
    return fail(AFD_ERR_NOT_CONVERGED, "buckling iteration did not reach tol %.3g in %d steps", tol, max_iter);
  return AFD_OK;
}

int afd_buckling_sensitivity(afd_mesh* m, float* out, int out_on_device) {
  if (!m || !out) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (!m->buckling_valid) return fail(AFD_ERR_STATE, "no buckling modes: call afd_buckling first");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  const Grid& g = m->gr;
  const int n = m->modal_n;
  TRY(upload_geo_table(m));
  float* dst = out_on_device ? out : m->fbuf;
  k_buckling_topo<<<dim3(grid_blocks(g.nelem, 256, 8 * RED_BLOCKS), n), 256, 0, m->s>>>(g, m->mX, m->bcoef, m->E64,
                                                                                        m->bS6, m->w64.K, dst);
  m->launches++;
  CK(cudaGetLastError());
  if (!out_on_device)
    CK(cudaMemcpyAsync(out, m->fbuf, (size_t)n * g.nelem * sizeof(float), cudaMemcpyDeviceToHost, m->s));
  return finish(m);
}

int afd_eigen_sensitivity(afd_mesh* m, float* out, int out_on_device) {
  if (!m || !out) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (!m->modal_valid) return fail(AFD_ERR_STATE, "no modes: call afd_modal first");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  const Grid& g = m->gr;
  FieldConsts F;
  const double nu = m->opt.nu;
  F.lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  F.mu = 1.0 / (2.0 * (1.0 + nu));
  F.nu = nu;
  F.inv4h = 1.0 / (4.0 * m->opt.h);
  const int n = m->modal_n;
  float* dst = out_on_device ? out : m->fbuf;   // fbuf holds >= modal block x N_e floats
  k_eigen_topo<<<dim3(grid_blocks(g.nelem, 256, 8 * RED_BLOCKS), n), 256, 0, m->s>>>(g, m->mX, m->mlam, m->E64, F,
                                                                                     m->modal_rho, dst); m->launches++;
  CK(cudaGetLastError());
  if (!out_on_device)
    CK(cudaMemcpyAsync(out, m->fbuf, (size_t)n * g.nelem * sizeof(float), cudaMemcpyDeviceToHost, m->s));
  return finish(m);
}

// Top-k selection on device keys (stream s); kept/E written on the device.
static int select_topk_dev(cudaStream_t s, const float* keys, int64_t n, int64_t k, uint8_t* kept, SelectState* st,
                           uint32_t* cnt, double* E64, float* E32, double e_void, float* tau, int64_t* nl) {
  SelectState init;
  memset(&init, 0, sizeof(init));
  init.kk = (uint64_t)k;
  CK(cudaMemcpyAsync(st, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  const int hb = (int)std::min<int64_t>((n + 255) / 256, 4 * RED_BLOCKS);
  if (k > 0) {
    for (int pass = 0; pass < 4; ++pass) {
      const int shift = 24 - 8 * pass;
      k_select_hist<<<std::max(hb, 1), 256, 0, s>>>(n, keys, st, shift); if (nl) ++*nl;
      k_select_pick<<<1, 32, 0, s>>>(st, shift); if (nl) ++*nl;
    }
  } else {
    // keep nothing: a cut above every key
    SelectState none = init;
    none.prefix = 0xffffffffu;
    none.kk = 0;
    CK(cudaMemcpyAsync(st, &none, sizeof(none), cudaMemcpyHostToDevice, s));
  }
  const int nch = (int)((n + SEL_CHUNK - 1) / SEL_CHUNK);
  if (nch > 0) {
    k_count_eq<<<nch, 256, 0, s>>>(n, keys, st, cnt); if (nl) ++*nl;
    k_scan_counts<<<1, 32, 0, s>>>(nch, cnt); if (nl) ++*nl;
    k_mark<<<nch, 256, 0, s>>>(n, keys, st, cnt, kept, E64, E32, e_void); if (nl) ++*nl;
  }
  CK(cudaGetLastError());
  SelectState fin;
  CK(cudaMemcpyAsync(&fin, st, sizeof(fin), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (tau) {
    if (k == 0) {
      *tau = NAN;
    } else {
      uint32_t kk = fin.prefix;
      uint32_t u = (kk & 0x80000000u) ? (kk & 0x7fffffffu) : ~kk;
      float f;
      memcpy(&f, &u, 4);
      *tau = f;
    }
  }
  return AFD_OK;
}

int afd_select_topk(const float* keys, int64_t n, int64_t k, uint8_t* kept, float* tau_out, void* cuda_stream) {
  if (n < 0 || k < 0 || k > n) return fail(AFD_ERR_INVALID_ARG, "need 0 <= k <= n");
  if (n > 0 && (!keys || !kept)) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (n == 0) {
    if (tau_out) *tau_out = NAN;
    return AFD_OK;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  SelectState* st = nullptr;
  uint32_t* cnt = nullptr;
  const int nch = (int)((n + SEL_CHUNK - 1) / SEL_CHUNK);
  TRY(dalloc(&st, 1));
  int rc = dalloc(&cnt, (size_t)nch);
  if (rc == AFD_OK) rc = select_topk_dev(s, keys, n, k, kept, st, cnt, nullptr, nullptr, 0.0, tau_out, nullptr);
  cudaFree(st);
  if (cnt) cudaFree(cnt);
  return rc;
}

// ---- afd_select_topk_noalloc: the top-k selection without device allocation ----
// Its scratch (the radix-select state, then one count per chunk of SEL_CHUNK
// keys) is a file-scope device array: every device that loads this library
// holds it until the process exits, and every call shares it.
constexpr int64_t NOALLOC_MAX_CHUNKS = 4096;
constexpr int64_t NOALLOC_MAX_KEYS = NOALLOC_MAX_CHUNKS * SEL_CHUNK;  // 16,777,216 keys
constexpr size_t NOALLOC_STATE_BYTES = (sizeof(SelectState) + 255) / 256 * 256;
constexpr size_t NOALLOC_BYTES = NOALLOC_STATE_BYTES + NOALLOC_MAX_CHUNKS * sizeof(uint32_t);
static __device__ __align__(256) unsigned char g_topk_scratch[NOALLOC_BYTES];

// Device address of g_topk_scratch on the current device.  Host code only
// holds a host-side stand-in for the symbol, so the address is looked up once
// per device (with that device current) and cached.
static int noalloc_scratch(void** out) {
  static std::mutex mu;
  static void* addr[128] = {nullptr};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(AFD_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_topk_scratch);
    if (e != cudaSuccess) return fail(AFD_ERR_CUDA, "cudaGetSymbolAddress(g_topk_scratch): %s", cudaGetErrorString(e));
    addr[dev] = p;
  }
  *out = addr[dev];
  return AFD_OK;
}

// Device that holds a device (or managed) pointer; refuses host memory.
static int device_of(const void* p, const char* what, int* dev) {
  cudaPointerAttributes at;
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(AFD_ERR_INVALID_ARG, "%s: not a CUDA pointer (%s)", what, cudaGetErrorString(e));
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(AFD_ERR_INVALID_ARG, "%s must be device memory", what);
  *dev = at.device;
  return AFD_OK;
}

int afd_select_topk_noalloc(const float* keys, int64_t n, int64_t k, uint8_t* kept, float* tau_out,
                            void* cuda_stream) {
  if (n < 0 || k < 0 || k > n) return fail(AFD_ERR_INVALID_ARG, "need 0 <= k <= n");
  if (n > NOALLOC_MAX_KEYS)
    return fail(AFD_ERR_INVALID_ARG, "afd_select_topk_noalloc takes at most %lld keys (got %lld)",
                (long long)NOALLOC_MAX_KEYS, (long long)n);
  if (n > 0 && (!keys || !kept)) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (n == 0) {
    if (tau_out) *tau_out = NAN;
    return AFD_OK;
  }
  // The scratch looked up below is the one of the keys' device: switch to it
  // for the call, and refuse `kept` on another device.
  int dk = 0, dm = 0;
  TRY(device_of(keys, "keys", &dk));
  TRY(device_of(kept, "kept", &dm));
  if (dk != dm) return fail(AFD_ERR_INVALID_ARG, "keys (device %d) and kept (device %d) on different devices", dk, dm);
  DeviceGuard guard(dk);
  void* base = nullptr;
  TRY(noalloc_scratch(&base));
  SelectState* st = (SelectState*)base;
  uint32_t* cnt = (uint32_t*)((unsigned char*)base + NOALLOC_STATE_BYTES);
  return select_topk_dev((cudaStream_t)cuda_stream, keys, n, k, kept, st, cnt, nullptr, nullptr, 0.0, tau_out, nullptr);
}

static int casting_args_ok(int nx, int ny, int nz, int axis, int parting) {
  if (axis < 0 || axis > 2) return fail(AFD_ERR_INVALID_ARG, "casting axis must be 0, 1 or 2");
  const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
  if (parting < 0 || parting > n) return fail(AFD_ERR_INVALID_ARG, "parting index must be in [0, %d]", n);
  return AFD_OK;
}

static int launch_casting_scan(cudaStream_t s, int nx, int ny, int nz, int axis, int parting, float* keys,
                               int64_t* launches) {
  const size_t nlines = axis == 0 ? (size_t)ny * nz : (axis == 1 ? (size_t)nx * nz : (size_t)nx * ny);
  if (axis == 0)
    k_casting_scan_x<<<(unsigned)((nlines + CASTX_L - 1) / CASTX_L), CASTX_T, 0, s>>>(nx, (int)nlines, parting, keys);
  else
    k_casting_scan_strided<<<grid_blocks(nlines, 128, 8192), 128, 0, s>>>(nx, ny, nz, axis, parting, keys);
  if (launches) ++*launches;
  CK(cudaGetLastError());
  return AFD_OK;
}

int afd_casting_scan(float* keys, int nx, int ny, int nz, int axis, int parting, void* cuda_stream) {
  if (!keys || nx < 1 || ny < 1 || nz < 1) return fail(AFD_ERR_INVALID_ARG, "bad argument");
  TRY(casting_args_ok(nx, ny, nz, axis, parting));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  TRY(launch_casting_scan(s, nx, ny, nz, axis, parting, keys, nullptr));
  CK(cudaStreamSynchronize(s));
  return AFD_OK;
}

static int levelset_update_impl(afd_mesh* m, int kind, const double* weights, double volume_fraction, int axis,
                                int parting, double* tau_out, uint8_t* kept_out);

int afd_levelset_update(afd_mesh* m, int kind, const double* weights, double volume_fraction, double* tau_out,
                        uint8_t* kept_out) {
  return levelset_update_impl(m, kind, weights, volume_fraction, -1, 0, tau_out, kept_out);
}

int afd_levelset_update_cast(afd_mesh* m, int kind, const double* weights, double volume_fraction, int axis,
                             int parting, double* tau_out, uint8_t* kept_out) {
  if (!m) return fail(AFD_ERR_INVALID_ARG, "null argument");
  TRY(casting_args_ok(m->gr.nx, m->gr.ny, m->gr.nz, axis, parting));
  return levelset_update_impl(m, kind, weights, volume_fraction, axis, parting, tau_out, kept_out);
}

static int ensure_select(afd_mesh* m) {
  const int64_t n = m->gr.nelem;
  if (!m->fkeys) {
    TRY(dalloc(&m->fkeys, (size_t)n));
    TRY(dalloc(&m->kept, (size_t)n));
    SelectState* st;
    TRY(dalloc(&st, 1));
    m->sel = st;
    TRY(dalloc(&m->selcnt, (size_t)((n + SEL_CHUNK - 1) / SEL_CHUNK)));
  }
  return AFD_OK;
}

// Back end of every level-set update: nf fields (field-major in `fields`,
// device) divided by their largest magnitude, weighted and added in float32
// (Eq. 3.17), the casting scan (axis >= 0), the cut at round(v N_e) (Eq. 3.6)
// and the new moduli.
static int levelset_cut(afd_mesh* m, const float* fields, int nf, const double* weights, double volume_fraction,
                        int axis, int parting, double* tau_out, uint8_t* kept_out, int64_t* k_out = nullptr) {
  const int64_t n = m->gr.nelem;
  TRY(ensure_select(m));
  float* dmaxv = m->fsmall + FS_MAXV;
  float* dw = m->fsmall + FS_WEIGHTS;
  TRY(maxabs_per_rhs(m, fields, nf, dmaxv));
  std::vector<float> wf(nf);
  for (int r = 0; r < nf; ++r) wf[r] = (float)weights[r];
  CK(cudaMemcpyAsync(dw, wf.data(), nf * sizeof(float), cudaMemcpyHostToDevice, m->s));
  k_combine<<<grid_blocks(n, 256, 4096), 256, 0, m->s>>>((int)n, nf, fields, dw, dmaxv, m->fkeys); m->launches++;
  CK(cudaGetLastError());
  if (axis >= 0) TRY(launch_casting_scan(m->s, m->gr.nx, m->gr.ny, m->gr.nz, axis, parting, m->fkeys, &m->launches));
  const double kd = std::floor(volume_fraction * (double)n + 0.5);
  const int64_t k = (int64_t)std::min<double>(std::max<double>(kd, 0.0), (double)n);
  float tau;
  TRY(select_topk_dev(m->s, m->fkeys, n, k, m->kept, (SelectState*)m->sel, m->selcnt, m->E64, nullptr, m->opt.e_void, &tau, &m->launches));
  TRY(refresh_moduli(m));
  if (kept_out) CK(cudaMemcpyAsync(kept_out, m->kept, (size_t)n, cudaMemcpyDeviceToHost, m->s));
  if (tau_out) *tau_out = (double)tau;
  if (k_out) *k_out = k;
  return finish(m);
}

static int levelset_update_impl(afd_mesh* m, int kind, const double* weights, double volume_fraction, int axis,
                                int parting, double* tau_out, uint8_t* kept_out) {
  if (!m || !weights) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (kind < 0 || kind > 2) return fail(AFD_ERR_INVALID_ARG, "unknown field kind %d", kind);
  if (!std::isfinite(volume_fraction)) return fail(AFD_ERR_INVALID_ARG, "volume fraction must be finite");
  if (!m->has_solution) return fail(AFD_ERR_STATE, "no solution");
  DeviceGuard dg(m->device);
  const int cached = m->fcache_kind;   // the field of the sensitivity call just before, if any
  TRY(enter(m));
  if (cached != kind) TRY(fields_to(m, kind, m->fbuf));
  return levelset_cut(m, m->fbuf, m->nrhs, weights, volume_fraction, axis, parting, tau_out, kept_out);
}

int afd_levelset_update_fields(afd_mesh* m, const float* fields, int fields_on_device, int nfields,
                               const double* weights, double volume_fraction, int axis, int parting, double* tau_out,
                               uint8_t* kept_out) {
  if (!m || !fields || !weights) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (nfields < 1 || nfields > MAX_RHS) return fail(AFD_ERR_INVALID_ARG, "nfields must be in [1, %d]", MAX_RHS);
  if (!std::isfinite(volume_fraction)) return fail(AFD_ERR_INVALID_ARG, "volume fraction must be finite");
  if (axis >= 0) TRY(casting_args_ok(m->gr.nx, m->gr.ny, m->gr.nz, axis, parting));
  if (!m->has_moduli) return fail(AFD_ERR_STATE, "moduli not set");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  const size_t need = (size_t)nfields * m->gr.nelem;
  if (need > m->lsbuf_cap) {
    dfree(m->lsbuf);
    m->lsbuf_cap = 0;
    TRY(dalloc(&m->lsbuf, need));
    m->lsbuf_cap = need;
  }
  CK(cudaMemcpyAsync(m->lsbuf, fields, need * sizeof(float),
                     fields_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->s));
  return levelset_cut(m, m->lsbuf, nfields, weights, volume_fraction, axis, parting, tau_out, kept_out);
}

// One y = K u launch for one vector in arithmetic `arith` (AFD_F32, AFD_F64 or AFD_F64_DF).
static int apply_one(afd_mesh* m, int arith, const void* u, void* y) {
  if (arith == AFD_F64)
    return launch_stencil<double, ST_APPLY, double>(m, (const double*)u, (double*)y, m->w64.E, nullptr, nullptr,
                                                    nullptr, nullptr, 1, m->w64.K);
  if (arith == AFD_F64_DF)
    return launch_stencil<double, ST_APPLY, double, dfloat>(m, (const double*)u, (double*)y, m->w64.E, nullptr,
                                                            nullptr, nullptr, nullptr, 1, m->w64.K);
  return launch_stencil<float, ST_APPLY, float>(m, (const float*)u, (float*)y, m->w32.E, nullptr, nullptr, nullptr,
                                                nullptr, 1, m->w32.K);
}

static bool valid_arith(int arith) { return arith == AFD_F32 || arith == AFD_F64 || arith == AFD_F64_DF; }

int afd_apply_stiffness(afd_mesh* m, int arith, int n_rhs, const void* u, void* y) {
  if (!m || !u || !y) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (n_rhs < 1) return fail(AFD_ERR_INVALID_ARG, "n_rhs must be >= 1");
  if (!m->has_moduli) return fail(AFD_ERR_STATE, "moduli not set");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  if (!valid_arith(arith)) return fail(AFD_ERR_INVALID_ARG, "arith must be AFD_F32, AFD_F64 or AFD_F64_DF");
  // caller arrays are RHS-major with stride ndof: one launch per RHS
  const size_t nd = (size_t)m->gr.ndof;
  const size_t es = arith == AFD_F32 ? sizeof(float) : sizeof(double);
  for (int r = 0; r < n_rhs; ++r)
    TRY(apply_one(m, arith, (const char*)u + r * nd * es, (char*)y + r * nd * es));
  return finish(m);
}

int afd_apply_search_direction(afd_mesh* m, int n_rhs, const float* z, const float* p_old, const double* mu,
                               const double* beta, float* p_out, float* q_out, double* pq_out) {
  if (!m || !z || !p_old || !mu || !beta || !p_out || !q_out) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (n_rhs < 1) return fail(AFD_ERR_INVALID_ARG, "n_rhs must be >= 1");
  if (!m->has_moduli || !m->has_loads) return fail(AFD_ERR_STATE, "set moduli and loads first");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  TRY(build_coarse(m));
  const size_t nd = (size_t)m->gr.ndof;
  const int nsb = stencil_blocks(m, false);
  TRY(ensure_partials(m, (size_t)nsb));
  std::vector<double> parts(nsb);
  for (int r = 0; r < n_rhs; ++r) {
    // beta reaches the kernel through the solver state of RHS 0 (the kernel
    // is launched for one RHS at a time on caller arrays of stride ndof)
    CGState h;
    memset(&h, 0, sizeof(h));
    h.beta = beta[r];
    CK(cudaMemcpyAsync(m->st, &h, sizeof(h), cudaMemcpyHostToDevice, m->s));
    TRY((launch_stencil<float, ST_APPLY_DOT, float>(m, p_old + r * nd, q_out + r * nd, m->w32.E, nullptr, nullptr,
                                                     m->partials, nullptr, 1, m->w32.K, m->st, nullptr, z + r * nd,
                                                     mu + (size_t)r * m->nc, p_out + r * nd, nullptr)));
    if (pq_out) {
      CK(cudaMemcpyAsync(parts.data(), m->partials, nsb * sizeof(double), cudaMemcpyDeviceToHost, m->s));
      CK(cudaStreamSynchronize(m->s));
      double sum = 0.0;
      for (int b = 0; b < nsb; ++b) sum += parts[b];
      pq_out[r] = sum;
    }
  }
  return finish(m);
}

int afd_deflation_wt(afd_mesh* m, int n_rhs, const double* v, double* out) {
  if (!m || !v || !out || n_rhs < 1) return fail(AFD_ERR_INVALID_ARG, "bad argument");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  for (int r = 0; r < n_rhs; ++r) {
    k_restrict<double><<<dim3(m->gp.ng, 1), 256, 0, m->s>>>(m->gr, m->gp, v + (size_t)r * m->gr.ndof, nullptr, m->fixed,
                                                            out + (size_t)r * m->nc, nullptr, nullptr); m->launches++;
  }
  CK(cudaGetLastError());
  return finish(m);
}

int afd_deflation_w(afd_mesh* m, int n_rhs, const double* y, double* out) {
  if (!m || !y || !out || n_rhs < 1) return fail(AFD_ERR_INVALID_ARG, "bad argument");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  for (int r = 0; r < n_rhs; ++r) {
    k_prolong<double><<<dim3(grid_blocks(m->gr.nnodes, 256, 4096), 1), 256, 0, m->s>>>(
        1, m->gr, m->gp, out + (size_t)r * m->gr.ndof, nullptr, y + (size_t)r * m->nc, m->fixed, nullptr); m->launches++;
  }
  CK(cudaGetLastError());
  return finish(m);
}

int afd_coarse_size(afd_mesh* m) { return m ? m->nc : 0; }

int64_t afd_kernel_launches(const afd_mesh* m) { return m ? m->launches : 0; }

int afd_stencil_depth(const afd_mesh* m) { return m ? m->kz32 : 0; }

int afd_stencil_warps(const afd_mesh* m) { return m ? m->ty32 : 0; }

int afd_stencil_async(const afd_mesh* m) { return m ? (m->async32 == 2 && m->rp32 ? 3 : m->async32) : 0; }

int afd_set_stencil_shape(afd_mesh* m, int warps, int planes, int async_staging) {
  if (!m || (warps != 8 && warps != 16) || planes < 1 || async_staging < 0 || async_staging > 3)
    return fail(AFD_ERR_INVALID_ARG, "warps must be 8 or 16, planes >= 1, async_staging 0, 1, 2 or 3");
  m->ty32 = warps;
  m->async32 = async_staging == 3 ? 2 : async_staging;
  m->rp32 = async_staging == 3 ? 1 : 0;
  m->kz32 = std::min(planes, m->gr.nnz);
  m->tuned = true;
  invalidate_graphs(m);
  return AFD_OK;
}

int afd_time_dpcg_kernels(afd_mesh* m, int iters, int nsplit, int variant, double* us_out5) {
  if (!m || !us_out5 || iters < 1 || iters > 4096 || nsplit < 0 || nsplit > 64 || variant < 0 || variant > 1)
    return fail(AFD_ERR_INVALID_ARG, "bad argument");
  if (!m->has_solution || m->opt.precision != AFD_MIXED || !m->w32.x || !m->coarse_valid)
    return fail(AFD_ERR_STATE, "needs a completed AFD_MIXED solve on this mesh");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  const int R = m->nrhs;
  const Grid& gr = m->gr;
  const int keep_split = m->nsplit;
  if (nsplit > 0) {
    TRY(ensure_cpart(m, nsplit));
    m->nsplit = nsplit;
  }
  // continue the last inner iteration without a stopping test
  std::vector<CGState> h(R);
  CK(cudaMemcpyAsync(h.data(), m->st, R * sizeof(CGState), cudaMemcpyDeviceToHost, m->s));
  CK(cudaStreamSynchronize(m->s));
  std::vector<int> hd(R, 0);
  for (int r = 0; r < R; ++r) {
    h[r].done = 0;
    h[r].status = 0;
    h[r].target2 = -1.0;
    h[r].max_iters = 1 << 30;
    if (!(h[r].rz > 0.0)) h[r].rz = 1.0;
    h[r].rzs[0] = h[r].rzs[1] = h[r].rz;
    h[r].its[0] = h[r].its[1] = 0;
  }
  CK(cudaMemcpyAsync(m->st, h.data(), R * sizeof(CGState), cudaMemcpyHostToDevice, m->s));
  CK(cudaMemcpyAsync(m->done, hd.data(), R * sizeof(int), cudaMemcpyHostToDevice, m->s));
  Work<float>& w = m->w32;
  const dim3 vg(RED_BLOCKS, R);
  const int crows = (m->nc * 32 + CSTEP_THREADS - 1) / CSTEP_THREADS;
  size_t csmem = 0;
  TRY(coarse_step_smem<float>(m, csmem));
  unsigned int* cnt_co = m->counters + MAX_RHS;
  float* P[2] = {w.p, w.t};
  const dim3 pg(grid_blocks(gr.nnodes, 256, 4 * RED_BLOCKS), R);
  // six events per iteration, all enqueued before one synchronisation, so that
  // the stream stays ahead of the GPU and each pair brackets its kernel only
  std::vector<cudaEvent_t> evs((size_t)iters * 6);
  for (auto& e : evs) CK(cudaEventCreate(&e));
  double acc[5] = {0, 0, 0, 0, 0};
  int rc = AFD_OK;
  for (int it = 0; it < iters && rc == AFD_OK; ++it) {
    float* pold = P[it & 1];
    float* pnew = P[(it + 1) & 1];
    cudaEvent_t* ev = evs.data() + (size_t)it * 6;
    cudaEventRecord(ev[5], m->s);
    if (variant == 1) {  // p = beta p + z + W mu in place, then the plain p.Kp stencil
      k_prolong<float><<<pg, 256, 0, m->s>>>(0, gr, m->gp, P[0], w.z, m->mu, m->fixed, m->st);
      m->launches++;
      pnew = P[0];
    }
    cudaEventRecord(ev[0], m->s);
    if (variant == 1)
      rc = launch_stencil<float, ST_DOT_PLAIN, float>(m, pnew, w.q, w.E, nullptr, nullptr, m->partials, m->done, R,
                                                     w.K, m->st, nullptr);
    else {
      const IterPartials ip{m->updred, crows, m->wr, crows, it & 1};
      rc = launch_stencil<float, ST_APPLY_DOT, float>(m, pold, w.q, w.E, nullptr, nullptr, m->partials, m->done, R,
                                                     w.K, m->st, nullptr, w.z, m->mu, pnew, &ip);
    }
    cudaEventRecord(ev[1], m->s);
    k_update<float><<<vg, RED_THREADS, 0, m->s>>>(gr.ndof, gr.vs, w.x, w.r, w.z, pnew, w.q, w.invd, m->upart, m->st,
                                                 m->partials, stencil_blocks(m, false, R), m->done);
    cudaEventRecord(ev[2], m->s);
    rc = launch_coarse_rhs<float>(m, w, m->nsplit, R, false);
    cudaEventRecord(ev[3], m->s);
    k_coarse_step<float><<<crows, CSTEP_THREADS, csmem, m->s>>>(m->nc, R, m->Einv32, m->mu, m->st, m->grec, m->wr, 1, m->done,
                                                     cnt_co, m->upart, RED_BLOCKS, m->updred);
    cudaEventRecord(ev[4], m->s);
    m->launches += 4;
  }
  if (rc == AFD_OK && cudaEventSynchronize(evs[(size_t)iters * 6 - 2]) != cudaSuccess)
    rc = fail(AFD_ERR_CUDA, "timing run failed");
  for (int it = 0; it < iters && rc == AFD_OK; ++it) {
    cudaEvent_t* ev = evs.data() + (size_t)it * 6;
    for (int q = 0; q < 4; ++q) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[q], ev[q + 1]);
      acc[q] += ms;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[5], ev[0]);
    acc[4] += ms;
  }
  for (auto& e : evs) cudaEventDestroy(e);
  for (int r = 0; r < R; ++r) hd[r] = 1;
  CK(cudaMemcpyAsync(m->done, hd.data(), R * sizeof(int), cudaMemcpyHostToDevice, m->s));
  m->nsplit = keep_split;
  invalidate_graphs(m);
  TRY(rc);
  for (int q = 0; q < 5; ++q) us_out5[q] = acc[q] * 1e3 / iters;
  return finish(m);
}

int afd_solver_phase_times(afd_mesh* m, double* out10, int reset) {
  if (!m || !out10) return fail(AFD_ERR_INVALID_ARG, "null argument");
  DeviceGuard dg(m->device);
  unsigned long long h[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (m->ptime) {
    CK(cudaMemcpyAsync(h, m->ptime, sizeof(h), cudaMemcpyDeviceToHost, m->s));
    if (reset) CK(cudaMemsetAsync(m->ptime, 0, sizeof(h), m->s));
    CK(cudaStreamSynchronize(m->s));
  }
  for (int q = 0; q < 10; ++q) out10[q] = q == 5 ? (double)h[q] : (double)h[q] * 1e-6;
  return AFD_OK;
}

size_t afd_mesh_bytes(int nx, int ny, int nz, int n_rhs, const afd_options* opt) {
  afd_options o;
  afd_default_options(&o);
  if (opt) o = *opt;
  if (nx < 1 || ny < 1 || nz < 1 || n_rhs < 1) return 0;
  const size_t ne = (size_t)nx * ny * nz;
  const size_t nn = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  const size_t vs = (3 * nn + 3) / 4 * 4;
  const int g = pick_group(nx, ny, nz, o.group);
  const size_t ng = (size_t)std::max(nx / g, 1) * std::max(ny / g, 1) * std::max(nz / g, 1);
  const size_t nc = 6 * ng;
  const bool f64 = o.precision == AFD_FP64;
  const size_t tsz = f64 ? 8 : 4;
  size_t b = 0;
  b += ne * (8 + 4) + ne * (4 * (size_t)n_rhs + 4 + 1);            // moduli, fields, keys, kept
  b += nn * (1 + 4 + (f64 ? 8 : 0)) + vs * (4 + (f64 ? 8 : 0));   // mask, Jacobi factors
  b += (size_t)n_rhs * vs * (2 * 8 + 8 * tsz);                      // f, u (FP64) + Krylov work
  b += nc * nc * (8 + tsz) + nc * GJ_NB * 2 * 8 + GJ_NB * GJ_NB * 8; // coarse matrix, inverse, sweep scratch
  if (!f64 && o.coarse_fp64) b += nc * nc * 8;                      // FP64 inverse before its FP32 rounding
  const size_t box = (size_t)(g + 3) * (g + 3) * (g + 3);
  if (f64 || o.persistent) b += ng * box * (18 * tsz + 4);          // K W on group shells (upper bound)
  else b += ng * (box - (size_t)std::max(g - 3, 0) * std::max(g - 3, 0) * std::max(g - 3, 0)) * 16;  // cut records
  b += (size_t)n_rhs * (nc * 4 * 8 + ng * 64 * 12 * 8) + 64 * 1024 * 1024 / 8;  // coarse vectors, partials
  return b + b / 10;
}

int afd_time_stiffness(afd_mesh* m, int arith, int n_rhs, const void* u, void* y, int launches, double* ms_out) {
  if (!m || !u || !y || !ms_out || launches < 1 || n_rhs < 1) return fail(AFD_ERR_INVALID_ARG, "bad argument");
  if (!m->has_moduli) return fail(AFD_ERR_STATE, "moduli not set");
  if (!valid_arith(arith)) return fail(AFD_ERR_INVALID_ARG, "arith must be AFD_F32, AFD_F64 or AFD_F64_DF");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, m->s));
  const size_t nd = (size_t)m->gr.ndof;
  const size_t es = arith == AFD_F32 ? sizeof(float) : sizeof(double);
  for (int i = 0; i < launches; ++i)
    for (int r = 0; r < n_rhs; ++r) TRY(apply_one(m, arith, (const char*)u + r * nd * es, (char*)y + r * nd * es));
  CK(cudaEventRecord(e1, m->s));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = (double)ms / launches;
  return finish(m);
}

int afd_coarse_inverse(afd_mesh* m, double* out_host) {
  if (!m || !out_host) return fail(AFD_ERR_INVALID_ARG, "null argument");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  m->coarse_valid = false;
  TRY(assemble_coarse(m));
  const size_t nn = (size_t)m->nc * m->nc;
  if (m->opt.precision == AFD_FP64 || m->opt.coarse_fp64) {
    if (!m->Einv64) TRY(dalloc(&m->Einv64, nn));
    TRY(scale_and_invert<double>(m, m->Einv64, 1e-12));
    CK(cudaMemcpyAsync(out_host, m->Einv64, nn * sizeof(double), cudaMemcpyDeviceToHost, m->s));
    TRY(finish(m));
  } else {
    if (!m->Einv32) TRY(dalloc(&m->Einv32, nn));
    TRY(scale_and_invert<float>(m, m->Einv32, 1e-6));
    std::vector<float> h(nn);
    CK(cudaMemcpyAsync(h.data(), m->Einv32, nn * sizeof(float), cudaMemcpyDeviceToHost, m->s));
    TRY(finish(m));
    for (size_t q = 0; q < nn; ++q) out_host[q] = h[q];
  }
  return AFD_OK;
}

int afd_coarse_matrix(afd_mesh* m, double* out_host) {
  if (!m || !out_host) return fail(AFD_ERR_INVALID_ARG, "null argument");
  DeviceGuard dg(m->device);
  TRY(enter(m));
  m->coarse_valid = false;
  TRY(assemble_coarse(m));
  CK(cudaMemcpyAsync(out_host, m->Ec, (size_t)m->nc * m->nc * sizeof(double), cudaMemcpyDeviceToHost, m->s));
  return finish(m);
}

// ---- augmented Lagrangian scalars (Eqs. 3.11, 3.12, 3.18) ----
void afd_al_init(afd_al_state* s) {
  if (!s) return;
  s->mu = 100.0;
  s->gamma = 10.0;
  s->g = 0.0;
  s->k = 0;
}

void afd_al_update(afd_al_state* s, double g_new) {
  if (!s) return;
  s->k += 1;
  s->mu = std::max(s->mu + s->gamma * g_new, 0.0);
  if (!(std::max(g_new, 0.0) <= 0.25 * std::max(s->g, 0.0))) s->gamma = std::max(10.0 * s->gamma, (double)s->k * s->k);
  s->g = g_new;
}

double afd_al_weight(const afd_al_state* s) {
  if (!s) return 0.0;
  const double w = s->mu + s->gamma * s->g;
  return w > 0.0 ? w : 0.0;
}


// ---- the algorithm of Sec. 3.8 (topology.h) ----
int afd_topology_run(const afd_topology_spec* spec, const afd_topology_ops* ops, void* ctx,
                     afd_topology_record* hist, int hist_cap, afd_topology_result* res) {
  if (!spec || !ops || !ops->analyse || !ops->save_feasible || !ops->restore_feasible || !ops->cut)
    return fail(AFD_ERR_INVALID_ARG, "null spec or callback");
  if (const char* why = topo_check(*spec)) return fail(AFD_ERR_INVALID_ARG, "%s", why);
  if (hist_cap < 0) return fail(AFD_ERR_INVALID_ARG, "hist_cap must be >= 0");
  auto call = [](int rc, const char* what) {
    if (rc != AFD_OK) fail(rc, "topology callback %s returned %d", what, rc);
    return rc;
  };
  return topology_loop(
      *spec,
      [&](int warm, double* v, int* it, double* rel) { return call(ops->analyse(ctx, warm, v, it, rel), "analyse"); },
      [&]() { return call(ops->save_feasible(ctx), "save_feasible"); },
      [&]() { return call(ops->restore_feasible(ctx), "restore_feasible"); },
      [&](const double* w, double v) { return call(ops->cut(ctx, w, v), "cut"); }, hist, hist_cap, res);
}

namespace {
// Device state of one run on a mesh: the fields of the active constraints
// (field-major, one slot each), and the last feasible design.
struct TopoMesh {
  afd_mesh* m = nullptr;
  int slot[AFD_CON_COUNT] = {-1, -1, -1, -1};
  int nf = 0;
  float* fields = nullptr;
  double* feasE = nullptr;
  uint8_t* feasKept = nullptr;
  bool cut_done = false;   // m->kept describes the current design
  ~TopoMesh() {
    dfree(fields);
    dfree(feasE);
    dfree(feasKept);
  }
};
}  // namespace

static int topo_mesh_analyse(TopoMesh& t, const afd_topology_spec& s, int warm, double* val, int* iters,
                             double* rel) {
  afd_mesh* m = t.m;
  const size_t ne = (size_t)m->gr.nelem;
  afd_stats st;
  TRY(afd_solve(m, s.tol, warm, &st, nullptr, 0));
  *iters = st.iters;
  *rel = st.rel_residual;
  TRY(afd_compliance(m, &val[AFD_CON_COMPLIANCE]));
  // the static fields first: the modal analysis discards the static solution
  if (t.slot[AFD_CON_COMPLIANCE] >= 0)
    TRY(afd_sensitivity(m, AFD_SENS_STRAIN_ENERGY, t.fields + t.slot[AFD_CON_COMPLIANCE] * ne, 1));
  if (t.slot[AFD_CON_STRESS] >= 0) {
    TRY(afd_pnorm_stress(m, s.p, &val[AFD_CON_STRESS]));
    afd_stats ast;
    TRY(afd_stress_sensitivity(m, s.p, s.tol, t.fields + t.slot[AFD_CON_STRESS] * ne, 1, &ast, nullptr, 0));
  }
  int it = 0, sit = 0;
  if (t.slot[AFD_CON_BUCKLING] >= 0) {   // the state is the solution just computed
    TRY(afd_buckling(m, 1, s.eig_tol, 100, &val[AFD_CON_BUCKLING], nullptr, 0, &it, &sit));
    TRY(afd_buckling_sensitivity(m, t.fields + t.slot[AFD_CON_BUCKLING] * ne, 1));
  }
  if (t.slot[AFD_CON_EIGEN] >= 0) {
    TRY(afd_modal(m, 1, s.rho, s.eig_tol, 100, &val[AFD_CON_EIGEN], nullptr, 0, &it, &sit));
    TRY(afd_eigen_sensitivity(m, t.fields + t.slot[AFD_CON_EIGEN] * ne, 1));
  }
  return AFD_OK;
}

int afd_constrained_topology(afd_mesh* m, const afd_topology_spec* spec, afd_topology_record* hist, int hist_cap,
                             afd_topology_result* res, uint8_t* kept_out, double* E_out) {
  if (!m || !spec) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (const char* why = topo_check(*spec)) return fail(AFD_ERR_INVALID_ARG, "%s", why);
  if (hist_cap < 0) return fail(AFD_ERR_INVALID_ARG, "hist_cap must be >= 0");
  if (!m->has_moduli || !m->has_loads) return fail(AFD_ERR_STATE, "set moduli and loads before the topology run");
  if (m->nrhs != 1) return fail(AFD_ERR_INVALID_ARG, "the topology run takes one load case (the mesh has %d)", m->nrhs);
  if (spec->casting_axis >= 0)
    TRY(casting_args_ok(m->gr.nx, m->gr.ny, m->gr.nz, spec->casting_axis, spec->casting_parting));
  DeviceGuard dg(m->device);
  TRY(enter(m));
  const afd_topology_spec& s = *spec;
  const size_t ne = (size_t)m->gr.nelem;
  TopoMesh t;
  t.m = m;
  for (int c = 0; c < AFD_CON_COUNT; ++c)
    if (topo_active(s, c)) t.slot[c] = t.nf++;
  TRY(dalloc(&t.fields, (size_t)t.nf * ne));
  TRY(dalloc(&t.feasE, ne));
  TRY(dalloc(&t.feasKept, ne));
  TRY(ensure_select(m));
  auto analyse = [&](int warm, double* v, int* it, double* rel) { return topo_mesh_analyse(t, s, warm, v, it, rel); };
  auto save = [&]() -> int {
    CK(cudaMemcpyAsync(t.feasE, m->E64, ne * sizeof(double), cudaMemcpyDeviceToDevice, m->s));
    if (t.cut_done)
      CK(cudaMemcpyAsync(t.feasKept, m->kept, ne, cudaMemcpyDeviceToDevice, m->s));
    else
      CK(cudaMemsetAsync(t.feasKept, 1, ne, m->s));
    return AFD_OK;
  };
  auto restore = [&]() -> int {
    TRY(afd_set_element_moduli(m, t.feasE, 1));
    CK(cudaMemcpyAsync(m->kept, t.feasKept, ne, cudaMemcpyDeviceToDevice, m->s));
    t.cut_done = true;
    return AFD_OK;
  };
  auto cut = [&](const double* w, double v) -> int {
    double wc[AFD_CON_COUNT];
    for (int c = 0; c < AFD_CON_COUNT; ++c)
      if (t.slot[c] >= 0) wc[t.slot[c]] = w[c];
    double tau;
    TRY(levelset_cut(m, t.fields, t.nf, wc, v, s.casting_axis, s.casting_parting, &tau, nullptr));
    t.cut_done = true;
    return AFD_OK;
  };
  TRY(topology_loop(s, analyse, save, restore, cut, hist, hist_cap, res));
  if (kept_out) CK(cudaMemcpyAsync(kept_out, t.feasKept, ne, cudaMemcpyDeviceToHost, m->s));
  if (E_out) CK(cudaMemcpyAsync(E_out, t.feasE, ne * sizeof(double), cudaMemcpyDeviceToHost, m->s));
  return finish(m);
}

int afd_volume_minimisation(afd_mesh* m, int steps, double dv, double j_factor, double tol, int kind,
                            afd_volmin_record* hist, uint8_t* kept_out, double* u_out) {
  if (!m || !hist) return fail(AFD_ERR_INVALID_ARG, "null argument");
  if (steps < 0 || !(dv > 0.0) || !(steps * dv < 1.0)) return fail(AFD_ERR_INVALID_ARG, "need steps >= 0 and 0 < steps dv < 1");
  if (!(j_factor > 0.0) || !(tol > 0.0)) return fail(AFD_ERR_INVALID_ARG, "j_factor and tol must be > 0");
  if (kind < 0 || kind > 2) return fail(AFD_ERR_INVALID_ARG, "unknown field kind %d", kind);
  if (!m->has_moduli || !m->has_loads) return fail(AFD_ERR_STATE, "set moduli and loads first");
  if (m->nrhs != 1) return fail(AFD_ERR_INVALID_ARG, "the volume minimisation takes one load case");
  DeviceGuard dg(m->device);
  using clk = std::chrono::steady_clock;
  auto t0 = clk::now();
  afd_stats st;
  TRY(afd_solve(m, tol, 0, &st, steps == 0 ? u_out : nullptr, 0));
  double J = 0.0;
  TRY(afd_compliance(m, &J));
  const double J0 = J, J_all = j_factor * J;
  afd_al_state al;
  afd_al_init(&al);
  const double nan = std::numeric_limits<double>::quiet_NaN();
  hist[0] = afd_volmin_record{0, 1.0, J, 1.0, J / J_all - 1.0, st.iters, st.rel_residual,
                              std::chrono::duration<double, std::milli>(clk::now() - t0).count(), nan,
                              afd_al_weight(&al), al.mu, al.gamma, (long long)m->gr.nelem};
  for (int k = 1; k <= steps; ++k) {
    t0 = clk::now();
    const double v = 1.0 - k * dv;
    const double w = afd_al_weight(&al);
    const bool last = k == steps;
    double tau = nan;
    int64_t kept = 0;
    TRY(enter(m));
    TRY(fields_to(m, kind, m->fbuf));
    TRY(levelset_cut(m, m->fbuf, 1, &w, v, -1, 0, &tau, last ? kept_out : nullptr, &kept));
    TRY(afd_solve(m, tol, 1, &st, last ? u_out : nullptr, 0));
    TRY(afd_compliance(m, &J));
    const double g = J / J_all - 1.0;
    afd_al_update(&al, g);
    hist[k] = afd_volmin_record{k, v, J, J / J0, g, st.iters, st.rel_residual,
                                std::chrono::duration<double, std::milli>(clk::now() - t0).count(), tau, w, al.mu,
                                al.gamma, (long long)kept};
  }
  return AFD_OK;
}

// Row-staged variant of the full-lattice stencil (FP32 vectors, EPI_D):
// neighbour spinors reach shared memory through bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier) instead of per-thread global
// loads.
//
// A tile is one X-row of output parity p: the n_X / 2 sites of parity p on
// the row (t, z, y), times all N right-hand sides, one thread per output
// (site j, RHS r).  With the even-odd compact index (lex / 2) and the
// RHS-innermost layout [group][Vh][N], every neighbour the row needs from the
// other parity lies in one of seven rows of that parity, and each such row is
// one contiguous range of hx * N 16-byte units per component group:
//   stage 0 / 1: rows t + 1 / t - 1  ->  the +T / -T hop
//   stage 2 / 3: rows z + 1 / z - 1  ->  the +Z / -Z hop
//   stage 4 / 5: rows y + 1 / y - 1  ->  the +Y / -Y hop
//   stage 6: the same row (t, z, y)  ->  the +X and -X hops
// The self-coupling term A(x) psi(x) starts the accumulator and beta = -1/2
// is folded into the sign of every hop.
// (on a row of parity p the site x = 2 j + xoff, xoff = (p + t + z + y) & 1;
// its Y, Z and T neighbours have the same compact position j, its X
// neighbours j and j +- 1 with wrap-around).  The self-coupling term and the
// links are read from global memory (links and blocks are shared by the N
// right-hand sides of a site, so L1 serves the repeats).
//
// Each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ... and streams
// their stages through a ring of D shared-memory slots: one thread issues the
// copies of stage k + D into the slot of stage k once every thread has
// finished stage k (block barrier, then a proxy fence), so D - 1 stages are in
// flight while one is consumed.  Waits on the mbarriers are bounded in time
// (`budget` clock cycles): on expiry the CTA records the failure in `err`,
// stops consuming, waits (again bounded) for the copies it has issued, and
// returns.  `poison` >= 0 names a stage of CTA 0 whose barrier is told to
// expect 16 bytes more than its copies deliver (every copy still lands), so
// that the expiry path can be tested.
#pragma once

#include <algorithm>
#include <cstdlib>

#include "dd_ops.h"

namespace dd {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Wait for phase `phase` of the barrier to complete, at most `budget` clock
// cycles; false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned phase, long long budget) {
  if (mbar_try_wait(bar, phase)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, phase)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned) completing on the barrier's transaction count.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

constexpr int kStages = 7;          // neighbour rows per tile
constexpr int kStageGroups = 6;     // FP32 spinor: six 16-byte groups
constexpr int kStageHeader = 128;   // bytes before the slots (barriers)
constexpr int kStageMaxSlots = 8;

// (t, z, y) of row index `row`, and the row index of a neighbour row
struct RowCoord {
  int t, z, y;
};

__device__ __forceinline__ RowCoord row_coord(const Geom& g, int row) {
  RowCoord c;
  c.y = row % g.n[2];
  const int r2 = row / g.n[2];
  c.z = r2 % g.n[1];
  c.t = r2 / g.n[1];
  return c;
}

__device__ __forceinline__ int stage_row(const Geom& g, const RowCoord& c, int st) {
  int t = c.t, z = c.z, y = c.y;
  switch (st) {
    case 0: t = t + 1 == g.n[0] ? 0 : t + 1; break;
    case 1: t = t == 0 ? g.n[0] - 1 : t - 1; break;
    case 2: z = z + 1 == g.n[1] ? 0 : z + 1; break;
    case 3: z = z == 0 ? g.n[1] - 1 : z - 1; break;
    case 4: y = y + 1 == g.n[2] ? 0 : y + 1; break;
    case 5: y = y == 0 ? g.n[2] - 1 : y - 1; break;
    default: break;
  }
  return (t * g.n[1] + z) * g.n[2] + y;
}

// Issue the copies of local stage k (tile k / 7 of this CTA, stage k % 7)
// into slot `slot`.  Tile tau: parity tau & 1 of row tau >> 1.
__device__ __forceinline__ void stage_issue(const HopArgs& a, int64_t k, float4* slot, uint64_t* bar, int hx,
                                            unsigned extra_tx = 0) {
  const int64_t tau = blockIdx.x + (k / kStages) * (int64_t)gridDim.x;
  const int st = (int)(k % kStages);
  const int p = (int)(tau & 1), q = p ^ 1;
  const RowCoord c = row_coord(a.g, (int)(tau >> 1));
  const int nrow = stage_row(a.g, c, st);
  const int64_t units = (int64_t)hx * a.nrhs;
  const unsigned bytes = (unsigned)(units * 16);
  mbar_arrive_expect_tx(bar, bytes * kStageGroups + extra_tx);
  const float4* src = reinterpret_cast<const float4*>(a.in[q].base) + (int64_t)nrow * units;
#pragma unroll
  for (int gr = 0; gr < kStageGroups; ++gr) bulk_copy_g2s(slot + gr * units, src + gr * a.gstride, bytes, bar);
}

// One hop of the output with the neighbour spinor at unit `u` of the slot
// (six groups of `units` 16-byte units) and the link already in registers.
template <int MU, int T, bool ADJ>
__device__ __forceinline__ void stage_hop_l(cx<float> acc[12], const float4* slot, int64_t units, int64_t u,
                                            const cx<float> lk[9], float sign) {
  cx<float> psi[12];
#pragma unroll
  for (int gr = 0; gr < kStageGroups; ++gr) {
    const float4 v = slot[gr * units + u];
    psi[2 * gr] = mk<float>(v.x, v.y);
    psi[2 * gr + 1] = mk<float>(v.z, v.w);
  }
  hop_regs<MU, T, ADJ, float>(acc, psi, lk, sign);
}

// MINB = 1: up to 512 threads, 128 registers; MINB = 3: up to 256 threads,
// 80 registers (three resident CTAs per SM).
template <int PG, bool DAG, int MINB>
__global__ void __launch_bounds__(MINB == 1 ? 512 : 256, MINB)
    k_hop_stage(const HopArgs a, int nslots, int64_t ntiles, int* err, long long budget, int poison) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  float4* slots = reinterpret_cast<float4*>(smem + kStageHeader);
  __shared__ int abort_flag;

  const int hx = a.g.n[3] >> 1;
  const int N = a.nrhs;
  const int64_t units = (int64_t)hx * N;
  const int64_t slot_units = units * kStageGroups;
  const int64_t Vh = a.g.Vh;
  const int o = threadIdx.x;
  const bool active = o < units;
  const int j = active ? o / N : 0;
  const int r = active ? o - j * N : 0;
  constexpr int TF = DAG ? +1 : -1;
  constexpr int TB = -TF;
  const float beta = (float)a.beta;

  const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t K = my_tiles * kStages;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int i = 0; i < nslots; ++i) mbar_init(&bar[i], 1);
    fence_barrier_init();
  }
  __syncthreads();
  int64_t issued = 0;
  if (threadIdx.x == 0) {
    for (; issued < K && issued < nslots; ++issued)
      stage_issue(a, issued, slots + (issued % nslots) * slot_units, &bar[issued % nslots], hx,
                  blockIdx.x == 0 && issued == poison ? 16u : 0u);
  }

  // Per tile: the links of a stage are loaded one stage ahead (before the
  // wait on the stage before), so their latency overlaps the staged data.
  int64_t k = 0;  // local stage counter
  bool aborted = false;
  for (int64_t it = 0; it < my_tiles && !aborted; ++it) {
    const int64_t tau = blockIdx.x + it * (int64_t)gridDim.x;
    const int p = (int)(tau & 1), q = p ^ 1;
    const int64_t row = tau >> 1;
    const RowCoord c = row_coord(a.g, (int)row);
    const int xoff = (p + c.t + c.z + c.y) & 1;
    const int64_t s = row * hx + j;
    const int64_t u = (int64_t)j * N + r;
    const int jf = xoff ? (j + 1 == hx ? 0 : j + 1) : j;  // +X neighbour
    const int jb = xoff ? j : (j == 0 ? hx - 1 : j - 1);  // -X neighbour
    const float sgf = c.t == a.g.n[0] - 1 ? beta * (float)a.g.t_bc : beta;
    const float sgb = c.t == 0 ? beta * (float)a.g.t_bc : beta;
    cx<float> acc[12];
    if (active) {
      // A(x) psi(x); the hops are added with beta folded into their signs
      cx<float> y[12];
      load_spinor<P32, float>(a.y[p], a.gstride, s * N + r, y);
      block_apply<PG, float>(a.M[p], s, Vh, y, acc);
    }
    cx<float> la[9], lb[9], lc[9];
    if (active) load_link<PG, float>(a.U[p], s, Vh, 0, la, a.recon);

// wait for local stage k, run BODY on its slot, release the slot
#define DD_STAGE_STEP(...)                                                               \
  {                                                                                      \
    const int slot_i = (int)(k % nslots);                                                \
    if (threadIdx.x == 0 &&                                                              \
        !mbar_wait_bounded(&bar[slot_i], (unsigned)((k / nslots) & 1), budget))          \
      abort_flag = 1;                                                                    \
    __syncthreads(); /* one thread polls; the block barrier publishes the data */        \
    const bool ok = abort_flag == 0;                                                     \
    if (ok && active) {                                                                  \
      const float4* sl = slots + slot_i * slot_units;                                    \
      __VA_ARGS__                                                                        \
    }                                                                                    \
    __syncthreads();                                                                     \
    if (abort_flag) {                                                                    \
      aborted = true;                                                                    \
      break;                                                                             \
    }                                                                                    \
    if (threadIdx.x == 0 && issued < K) {                                                \
      fence_proxy_async_smem();                                                          \
      stage_issue(a, issued, slots + (issued % nslots) * slot_units, &bar[issued % nslots], hx); \
      ++issued;                                                                          \
    }                                                                                    \
    ++k;                                                                                 \
  }

    do {
      if (active) load_link<PG, float>(a.U[q], (int64_t)stage_row(a.g, c, 1) * hx + j, Vh, 0, lb, a.recon);
      DD_STAGE_STEP(stage_hop_l<0, TF, false>(acc, sl, units, u, la, sgf);)
      if (active) load_link<PG, float>(a.U[p], s, Vh, 1, la, a.recon);
      DD_STAGE_STEP(stage_hop_l<0, TB, true>(acc, sl, units, u, lb, sgb);)
      if (active) load_link<PG, float>(a.U[q], (int64_t)stage_row(a.g, c, 3) * hx + j, Vh, 1, lb, a.recon);
      DD_STAGE_STEP(stage_hop_l<1, TF, false>(acc, sl, units, u, la, beta);)
      if (active) load_link<PG, float>(a.U[p], s, Vh, 2, la, a.recon);
      DD_STAGE_STEP(stage_hop_l<1, TB, true>(acc, sl, units, u, lb, beta);)
      if (active) load_link<PG, float>(a.U[q], (int64_t)stage_row(a.g, c, 5) * hx + j, Vh, 2, lb, a.recon);
      DD_STAGE_STEP(stage_hop_l<2, TF, false>(acc, sl, units, u, la, beta);)
      if (active) {
        load_link<PG, float>(a.U[p], s, Vh, 3, la, a.recon);
        load_link<PG, float>(a.U[q], row * hx + jb, Vh, 3, lc, a.recon);
      }
      DD_STAGE_STEP(stage_hop_l<2, TB, true>(acc, sl, units, u, lb, beta);)
      DD_STAGE_STEP(stage_hop_l<3, TF, false>(acc, sl, units, (int64_t)jf * N + r, la, beta);
                    stage_hop_l<3, TB, true>(acc, sl, units, (int64_t)jb * N + r, lc, beta);
                    store_spinor<P32, float>(a.out[p], a.gstride, s * N + r, acc);)
    } while (false);
#undef DD_STAGE_STEP
  }
  if (aborted && threadIdx.x == 0) {
    atomicExch(err, 1);
    // let the copies already issued land before the CTA's shared memory goes
    for (int64_t k = issued - nslots < 0 ? 0 : issued - nslots; k < issued; ++k)
      mbar_wait_bounded(&bar[k % nslots], (unsigned)((k / nslots) & 1), budget);
  }
}

}  // namespace dd

namespace dd {

// Host side: launch the row-staged stencil for a full-lattice D / D^H apply
// with FP32 vectors when its shapes fit (one X-row of outputs per CTA, at
// most 512 threads; at least two stage slots in shared memory; 16-byte
// aligned fields).  Returns false (nothing launched) otherwise.
// Off unless DD_STAGE=1: measured on the GB300 it is about twice slower
// than the per-thread-load kernels (48^3 x 96: 3.2 vs 1.4 ms; 32^4 x 12 RHS:
// 2.5 vs 1.1 ms).  DD_STAGE_SLOTS sets the ring depth (default 4).
inline int stage_env(const char* name, int dflt) {
  const char* e = getenv(name);
  return e ? atoi(e) : dflt;
}

template <int PG>
bool launch_stage(const HopArgs& a, bool dagger, cudaStream_t st, cudaError_t* err_out) {
  static const int enabled = stage_env("DD_STAGE", 0);
  static const int want_slots = stage_env("DD_STAGE_SLOTS", 4);
  // DD_STAGE_WAIT_TEST=1 (tests of the expiry path): the first stage of CTA 0
  // expects 16 bytes more than its copies deliver, so that wait can only
  // expire; the wait budget drops from about 2 s to 0.1 s.
  static const int wait_test = stage_env("DD_STAGE_WAIT_TEST", 0);
  if (!enabled || a.npar != 2 || a.g.t0 != 0 || a.g.nt != a.g.n[0]) return false;
  const int hx = a.g.n[3] / 2;
  const int64_t units = (int64_t)hx * a.nrhs;
  if (units < 1 || units > 512) return false;
  for (int p = 0; p < 2; ++p)
    if (((uintptr_t)a.in[p].base & 15) || ((uintptr_t)a.y[p].base & 15) || ((uintptr_t)a.out[p].base & 15))
      return false;
  const size_t slot_bytes = (size_t)units * kStageGroups * 16;
  const size_t max_smem = 200 * 1024;
  int nslots = want_slots < 2 ? 2 : want_slots > kStageMaxSlots ? kStageMaxSlots : want_slots;
  while (nslots > 2 && kStageHeader + nslots * slot_bytes > max_smem) --nslots;
  const size_t smem = kStageHeader + nslots * slot_bytes;
  if (smem > max_smem) return false;
  static const int narrow_ok = stage_env("DD_STAGE_NARROW", 0);  // spills; measured slower
  const int threads = (int)((units + 31) / 32 * 32);
  const bool narrow = narrow_ok && threads <= 256;
  auto kern = narrow ? (dagger ? k_hop_stage<PG, true, 3> : k_hop_stage<PG, false, 3>)
                     : (dagger ? k_hop_stage<PG, true, 1> : k_hop_stage<PG, false, 1>);
  static bool configured[2][2] = {{false, false}, {false, false}};
  if (!configured[narrow][dagger]) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem) != cudaSuccess)
      return false;
    configured[narrow][dagger] = true;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
    return false;
  const int64_t ntiles = 2 * (int64_t)a.g.n[0] * a.g.n[1] * a.g.n[2];
  const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
  int* flag = device_error_flag();
  if (!flag) return false;
  kern<<<(unsigned)grid, threads, smem, st>>>(a, nslots, ntiles, flag, wait_test ? 200000000LL : 4000000000LL,
                                                wait_test ? 0 : -1);
  *err_out = cudaGetLastError();
  return true;
}

}  // namespace dd

// Batched apply of D over lattices of different sizes in one launch.
//
// Work items are tiles of `tile` consecutive (site, right-hand side) output
// slots of one lattice; with the RHS-innermost layout a tile covers
// tile / N sites times all N right-hand sides (the RHS block), so the links
// and self-coupling blocks of a site are fetched once for all its RHS from
// L1/L2.  The kernel walks the item list with a static stride of gridDim:
// in the persistent shape the grid is the resident CTA count (a multiple of
// the SM count) and every CTA loops over many items; in the flat shape the
// grid has one CTA per item.  There are no atomics, barriers or waits; each
// thread finds its lattice in the item prefix table.  A third shape launches
// every lattice with its own best single-lattice kernel (one thread per site
// and RHS, or blocks of 2 or 4 RHS, each with its own register allocation) on
// forked streams joined again at the end, which a CUDA graph captures as
// parallel branches.  The autotuner (dd_batch_tune) times tile sizes and all
// three shapes, and the chosen launch can be captured once in a CUDA graph
// and replayed.
#include <algorithm>
#include <vector>

#include "dd_hop.cuh"
#include "dd_internal.h"

struct dd_batch {
  std::vector<dd_clover*> ops;
  std::vector<int> nrhs;
  int prec = 0;
  int count = 0;
  int tile = 128;
  int ctas_per_sm = 4;
  int sms = 0;
  // DD_LAYOUT_NATIVE_PAIRED: lattices with an even RHS count take paired-RHS
  // fields (one launch per lattice only)
  int layout = DD_LAYOUT_NATIVE;
  dd::DevBuf args, item_start;
  dd::HopArgs* h_args = nullptr;  // pinned staging
  std::vector<const void*> last_in;
  std::vector<void*> last_out;
  int64_t total_items = 0;
  int staged_tile = -1;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  std::vector<const void*> g_in;
  std::vector<void*> g_out;
  // the per-lattice shape (ctas_per_sm == -1): forked streams and events,
  // lattices in decreasing order of work
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;
  std::vector<int> order;
  ~dd_batch() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (h_args) cudaFreeHost(h_args);
    for (cudaStream_t q : side) cudaStreamDestroy(q);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

namespace dd {

namespace {

// Resident CTAs asked of the compiler: about 168 registers per thread for 64
// and 128 threads (the RHS-blocked body holds two sets of accumulators; fewer
// registers spill hundreds of bytes), 128 for 256 threads.
template <int THREADS>
struct BatchMinBlocks {
  static constexpr int value = THREADS >= 256 ? 2 : 384 / THREADS;
};

template <int P, int THREADS>
__global__ void __launch_bounds__(THREADS, BatchMinBlocks<THREADS>::value)
    k_hop_batch(const HopArgs* __restrict__ args, const int64_t* __restrict__ item_start, int count,
                int64_t total_items) {
  int l = 0;
  for (int64_t item = blockIdx.x; item < total_items; item += gridDim.x) {
    while (l + 1 < count && item >= item_start[l + 1]) ++l;  // items only grow within a CTA
    const HopArgs& a = args[l];
    const int64_t tid = (item - item_start[l]) * THREADS + threadIdx.x;
    if (tid < (int64_t)a.g.Vh * ((a.nrhs + a.rhs_block - 1) / a.rhs_block) * a.npar) {
      if (a.rhs_block == 2)
        hop_thread_rb<P, P, P, false, EPI_D, 2>(a, tid);
      else
        hop_thread<P, P, P, false, EPI_D>(a, tid);
    }
  }
}

int stage(dd_batch* b, const void* const* ins, void* const* outs, cudaStream_t st) {
  bool same = b->staged_tile == b->tile && (int)b->last_in.size() == b->count;
  for (int i = 0; same && i < b->count; ++i) same = b->last_in[i] == ins[i] && b->last_out[i] == outs[i];
  if (same) return DD_OK;
  DD_CUDA(cudaStreamSynchronize(st));  // the staging buffer may still be in flight
  std::vector<int64_t> starts(b->count + 1, 0);
  const int pi = prec_index(b->prec);
  for (int i = 0; i < b->count; ++i) {
    const dd_clover* op = b->ops[i];
    const dd_lattice* lat = op->lat;
    HopArgs& a = b->h_args[i];
    a.g = lat->geom();
    a.g.zblock = zblock_for(lat->dims, stencil_bytes_per_site(b->prec, b->nrhs[i]));
    a.rhs_block = rb_worth(b->nrhs[i]) ? 2 : 1;
    prepare_divs(a.g);
    a.fblk = make_fastdiv((uint32_t)((b->nrhs[i] + a.rhs_block - 1) / a.rhs_block));
    a.nrhs = b->nrhs[i];
    a.p0 = 0;
    a.npar = 2;
    a.gstride = lat->Vh * b->nrhs[i];
    Field fi = field_view(lat, b->prec, 0, const_cast<void*>(ins[i]), b->nrhs[i]);
    Field fo = field_view(lat, b->prec, 0, outs[i], b->nrhs[i]);
    for (int p = 0; p < 2; ++p) {
      a.in[p] = fi.h[p];
      a.y[p] = fi.h[p];
      a.out[p] = fo.h[p];
      a.z[p] = HalfField{nullptr, nullptr};
      a.U[p] = op->gauge->U(pi, p);
      a.M[p] = op->M(pi, p);
    }
    a.beta = -0.5;
    a.recon = 0;  // three-row links (the batch carries several RHS per lattice)
    const int64_t slots = 2 * lat->Vh * ((b->nrhs[i] + a.rhs_block - 1) / a.rhs_block);
    starts[i + 1] = starts[i] + (slots + b->tile - 1) / b->tile;
  }
  b->total_items = starts[b->count];
  DD_CUDA(cudaMemcpyAsync(b->args.ptr, b->h_args, sizeof(HopArgs) * b->count, cudaMemcpyHostToDevice, st));
  DD_CUDA(cudaMemcpyAsync(b->item_start.ptr, starts.data(), sizeof(int64_t) * (b->count + 1),
                          cudaMemcpyHostToDevice, st));
  DD_CUDA(cudaStreamSynchronize(st));
  b->last_in.assign(ins, ins + b->count);
  b->last_out.assign(outs, outs + b->count);
  b->staged_tile = b->tile;
  return DD_OK;
}

template <int P, int T>
void launch_t(dd_batch* b, unsigned grid, cudaStream_t st) {
  k_hop_batch<P, T><<<grid, T, 0, st>>>(reinterpret_cast<const HopArgs*>(b->args.ptr),
                                        reinterpret_cast<const int64_t*>(b->item_start.ptr), b->count,
                                        b->total_items);
}

// every lattice with its own kernel on a forked stream, joined back into st
int launch_per_lattice(dd_batch* b, cudaStream_t st) {
  if (b->side.empty()) {
    b->side.resize(b->count);
    b->ev.resize(b->count + 1);
    for (int i = 0; i < b->count; ++i) DD_CUDA(cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking));
    for (int i = 0; i <= b->count; ++i) DD_CUDA(cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming));
  }
  DD_CUDA(cudaEventRecord(b->ev[b->count], st));
  for (int k = 0; k < b->count; ++k) {
    const int i = b->order[k];
    dd_clover* op = b->ops[i];
    const int paired = b->layout == DD_LAYOUT_NATIVE_PAIRED && b->nrhs[i] % 2 == 0;
    Field fi = field_view(op->lat, b->prec, 0, const_cast<void*>(b->last_in[i]), b->nrhs[i], paired);
    Field fo = field_view(op->lat, b->prec, 0, b->last_out[i], b->nrhs[i], paired);
    DD_CUDA(cudaStreamWaitEvent(b->side[k], b->ev[b->count], 0));
    DD_TRY(op_D(op, b->prec, b->prec, false, fi, fo, b->side[k]));
    DD_CUDA(cudaEventRecord(b->ev[k], b->side[k]));
  }
  for (int k = 0; k < b->count; ++k) DD_CUDA(cudaStreamWaitEvent(st, b->ev[k], 0));
  return DD_OK;
}

// ctas_per_sm == 0 selects the flat shape (one CTA per item), -1 the
// per-lattice shape.
int launch(dd_batch* b, cudaStream_t st) {
  if (b->ctas_per_sm < 0) return launch_per_lattice(b, st);
  const int64_t g = b->ctas_per_sm > 0 ? (int64_t)b->sms * b->ctas_per_sm : b->total_items;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, b->total_items));
  if (b->prec == P32) {
    if (b->tile == 64) launch_t<P32, 64>(b, grid, st);
    else if (b->tile == 256) launch_t<P32, 256>(b, grid, st);
    else launch_t<P32, 128>(b, grid, st);
  } else {
    if (b->tile == 64) launch_t<P16, 64>(b, grid, st);
    else if (b->tile == 256) launch_t<P16, 256>(b, grid, st);
    else launch_t<P16, 128>(b, grid, st);
  }
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

template <int P, int T>
int occupancy_t() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_hop_batch<P, T>, T, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    return 1;
  }
  return std::max(1, n);
}

int max_ctas(int prec, int tile) {
  if (prec == P32) return tile == 64 ? occupancy_t<P32, 64>() : tile == 256 ? occupancy_t<P32, 256>() : occupancy_t<P32, 128>();
  return tile == 64 ? occupancy_t<P16, 64>() : tile == 256 ? occupancy_t<P16, 256>() : occupancy_t<P16, 128>();
}

void drop_graph(dd_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
}

}  // namespace

}  // namespace dd

using namespace dd;

extern "C" {

int dd_batch_create(dd_clover* const* ops, int count, int prec, const int* nrhs, dd_batch** out) {
  if (!ops || !nrhs || !out || count < 1) return fail(DD_ERR_ARG, "null argument or empty batch");
  if (prec != DD_PREC_F32 && prec != DD_PREC_F16) return fail(DD_ERR_ARG, "batched precision must be F32 or F16");
  const int pi = prec_index(prec);
  for (int i = 0; i < count; ++i) {
    if (!ops[i] || nrhs[i] < 1) return fail(DD_ERR_ARG, "null operator or nrhs < 1");
    if (!ops[i]->clov[pi].ptr || !ops[i]->gauge->links[pi].ptr)
      return fail(DD_ERR_UNSUPPORTED, "precision not created in an operator of the batch");
  }
  dd_batch* b = new dd_batch;
  b->ops.assign(ops, ops + count);
  b->nrhs.assign(nrhs, nrhs + count);
  b->order.resize(count);
  for (int i = 0; i < count; ++i) b->order[i] = i;
  std::sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    return ops[x]->lat->V * (int64_t)nrhs[x] > ops[y]->lat->V * (int64_t)nrhs[y];
  });
  b->prec = prec;
  b->count = count;
  int dev = 0;
  int s = DD_OK;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev))
    s = cuda_fail(cudaGetLastError(), "device query");
  if (s == DD_OK) s = b->args.alloc(sizeof(HopArgs) * count);
  if (s == DD_OK) s = b->item_start.alloc(sizeof(int64_t) * (count + 1));
  if (s == DD_OK && cudaMallocHost((void**)&b->h_args, sizeof(HopArgs) * count) != cudaSuccess) {
    b->h_args = nullptr;
    s = fail(DD_ERR_OOM, "pinned host allocation failed");
  }
  if (s == DD_OK) b->ctas_per_sm = max_ctas(prec, b->tile);
  if (s != DD_OK) {
    delete b;
    return s;
  }
  *out = b;
  return DD_OK;
}

int dd_batch_set_layout(dd_batch* b, int layout) {
  if (!b) return fail(DD_ERR_ARG, "null batch");
  if (layout != DD_LAYOUT_NATIVE && layout != DD_LAYOUT_NATIVE_PAIRED)
    return fail(DD_ERR_ARG, "batch layout: DD_LAYOUT_NATIVE or DD_LAYOUT_NATIVE_PAIRED");
  b->layout = layout;
  if (layout == DD_LAYOUT_NATIVE_PAIRED) b->ctas_per_sm = -1;
  drop_graph(b);
  b->staged_tile = -1;
  return DD_OK;
}

int dd_batch_destroy(dd_batch* b) {
  delete b;
  return DD_OK;
}

int dd_apply_batched(dd_batch* b, const void* const* ins, void* const* outs, void* stream) {
  if (!b || !ins || !outs) return fail(DD_ERR_ARG, "null argument");
  for (int i = 0; i < b->count; ++i)
    if (!ins[i] || !outs[i]) return fail(DD_ERR_ARG, "null field pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DD_TRY(stage(b, ins, outs, st));
  return launch(b, st);
}

int dd_batch_tune(dd_batch* b, const void* const* ins, void* const* outs, void* stream, int* chosen3) {
  if (!b || !ins || !outs) return fail(DD_ERR_ARG, "null argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  DD_CUDA(cudaEventCreate(&e0));
  DD_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_tile = b->tile, best_ctas = b->ctas_per_sm;
  const int tiles[3] = {64, 128, 256};
  for (int ti = 0; ti < 3; ++ti) {
    const int cap = max_ctas(b->prec, tiles[ti]);
    // persistent shapes at full and reduced residency, the flat shape, and
    // (once) one launch per lattice
    const int shapes[5] = {cap, std::max(1, cap - 1), std::max(1, cap / 2), 0, -1};
    for (int ci = 0; ci < (ti == 0 ? 5 : 4); ++ci) {
      if (b->layout == DD_LAYOUT_NATIVE_PAIRED && shapes[ci] != -1) continue;  // paired fields: per lattice only
      b->tile = tiles[ti];
      b->ctas_per_sm = shapes[ci];
      DD_TRY(stage(b, ins, outs, st));
      DD_TRY(launch(b, st));  // warm-up
      DD_CUDA(cudaEventRecord(e0, st));
      for (int r = 0; r < 3; ++r) DD_TRY(launch(b, st));
      DD_CUDA(cudaEventRecord(e1, st));
      DD_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      DD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_tile = b->tile;
        best_ctas = b->ctas_per_sm;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tile = best_tile;
  b->ctas_per_sm = best_ctas;
  drop_graph(b);
  DD_TRY(stage(b, ins, outs, st));
  if (chosen3) {
    chosen3[0] = b->tile;
    chosen3[1] = b->tile;
    chosen3[2] = b->ctas_per_sm;
  }
  return DD_OK;
}

int dd_apply_batched_graph(dd_batch* b, const void* const* ins, void* const* outs, void* stream) {
  if (!b || !ins || !outs) return fail(DD_ERR_ARG, "null argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (b->gexec) {
    bool same = (int)b->g_in.size() == b->count;
    for (int i = 0; same && i < b->count; ++i) same = b->g_in[i] == ins[i] && b->g_out[i] == outs[i];
    if (!same) return fail(DD_ERR_ARG, "graph was captured with other field pointers");
    DD_CUDA(cudaGraphLaunch(b->gexec, st));
    return DD_OK;
  }
  DD_TRY(stage(b, ins, outs, st));
  cudaStream_t cap;
  DD_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  int s = DD_OK;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    s = cuda_fail(cudaGetLastError(), "cudaStreamBeginCapture");
  if (s == DD_OK) s = launch(b, cap);
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(cap, &g) != cudaSuccess && s == DD_OK) s = cuda_fail(cudaGetLastError(), "capture");
  if (s == DD_OK && cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess)
    s = cuda_fail(cudaGetLastError(), "cudaGraphInstantiate");
  cudaStreamDestroy(cap);
  if (s != DD_OK) {
    if (g) cudaGraphDestroy(g);
    b->gexec = nullptr;
    return s;
  }
  b->graph = g;
  b->g_in.assign(ins, ins + b->count);
  b->g_out.assign(outs, outs + b->count);
  DD_CUDA(cudaGraphLaunch(b->gexec, st));
  return DD_OK;
}

}  // extern "C"

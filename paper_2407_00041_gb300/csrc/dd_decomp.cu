// Domain decomposition on one GPU: the lattice of an operator handle split
// into grid[0] x grid[1] x grid[2] x grid[3] hyper-rectangular local lattices
// (Section 2.1 of the thesis), each owned by a virtual rank with its own
// links, self-coupling blocks, fields and face buffers, and the neighbour
// coupling evaluated as Algorithm 3 does: project and send the seams, compute
// the interior while the messages travel, then finish the boundary sites.
// A message is a plain device-to-device copy from the sender's outgoing
// buffer into the receiver's own incoming buffer, on a stream of its own.
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "dd_blas.h"
#include "dd_decomp.h"
#include "dd_internal.h"

using namespace dd;

struct dd_decomp {
  struct Rank {
    dd_lattice lat;
    dd_gauge gauge;
    dd_clover clov;
    int coord[4] = {0, 0, 0, 0};
    int off[4] = {0, 0, 0, 0};
    int lo[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};  // ranks at -mu and +mu
    DevBuf fin, fout, ftmp;  // native fields (full-lattice layout: even half, then odd half)
    DevBuf faces;            // [mu][lam_send, chi_send, lam_recv, chi_recv] messages
    DevBuf bsites;           // boundary sites, parity 0 then parity 1 (p * Vh + s)
    int64_t nb[2] = {0, 0};
    size_t msg[4] = {0, 0, 0, 0};  // bytes of one message of direction mu (current precision, RHS count)
    void* buf(int mu, int k) {
      size_t o = 0;
      for (int m = 0; m < mu; ++m) o += 4 * msg[m];
      return reinterpret_cast<char*>(faces.ptr) + o + k * msg[mu];
    }
  };
  const dd_clover* op = nullptr;
  int grid[4] = {1, 1, 1, 1};
  int local[4] = {0, 0, 0, 0};
  std::vector<std::unique_ptr<Rank>> ranks;
  cudaStream_t comm = nullptr;
  cudaEvent_t ev_pack = nullptr, ev_comm = nullptr;
  int field_prec = 0, field_nrhs = 0;  // shape of the rank fields since the last scatter
  ~dd_decomp() {
    if (ev_pack) cudaEventDestroy(ev_pack);
    if (ev_comm) cudaEventDestroy(ev_comm);
    if (comm) cudaStreamDestroy(comm);
  }
};

namespace {

struct SiteMap {
  int nl[4];    // local extents
  int off[4];   // offset of the rank
  int ng[4];    // global extents
  int64_t Vhl, Vhg;
};

// Global compact index of local site (p, s).
__device__ __forceinline__ int64_t global_site(const SiteMap& m, int p, int64_t s) {
  const int64_t lex2 = 2 * s;
  const int64_t row = lex2 / m.nl[3];
  const int x0 = (int)(lex2 - row * m.nl[3]);
  const int y = (int)(row % m.nl[2]);
  const int64_t r2 = row / m.nl[2];
  const int z = (int)(r2 % m.nl[1]);
  const int t = (int)(r2 / m.nl[1]);
  const int x = x0 + ((p ^ (t + z + y)) & 1);
  const int64_t g =
      (((int64_t)(t + m.off[0]) * m.ng[1] + (z + m.off[1])) * m.ng[2] + (y + m.off[2])) * m.ng[3] + (x + m.off[3]);
  return g >> 1;
}

// Arrays [G][Vh][W] of T, one parity: local <-> global (to_local = 1 copies
// global -> local).
template <typename T>
__global__ void k_dom_copy(SiteMap m, int p, const T* src, T* dst, int G, int W, int to_local) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m.Vhl * W) return;
  const int64_t sl = t / W;
  const int w = (int)(t - sl * W);
  const int64_t sg = global_site(m, p, sl);
  for (int g = 0; g < G; ++g) {
    const int64_t il = ((int64_t)g * m.Vhl + sl) * W + w, ig = ((int64_t)g * m.Vhg + sg) * W + w;
    if (to_local)
      dst[il] = src[ig];
    else
      dst[ig] = src[il];
  }
}

template <typename T>
int dom_copy(const SiteMap& m, int p, const void* src, void* dst, int G, int W, int to_local, cudaStream_t st) {
  const int64_t n = m.Vhl * W;
  if (n == 0) return DD_OK;
  k_dom_copy<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m, p, reinterpret_cast<const T*>(src),
                                                               reinterpret_cast<T*>(dst), G, W, to_local);
  DD_CUDA(cudaGetLastError());
  return DD_OK;
}

SiteMap site_map(const dd_decomp* D, const dd_decomp::Rank& r) {
  SiteMap m;
  for (int i = 0; i < 4; ++i) {
    m.nl[i] = r.lat.dims[i];
    m.off[i] = r.off[i];
    m.ng[i] = D->op->lat->dims[i];
  }
  m.Vhl = r.lat.Vh;
  m.Vhg = D->op->lat->Vh;
  return m;
}

// 16-byte groups per parity of a link or block array of precision index pi
int groups36(int pi) { return pi == 0 ? 36 : pi == 1 ? 18 : 9; }

int spinor_groups(int prec) { return prec == P64 ? 12 : prec == P32 ? 6 : 3; }

// The rank's copy of the global handles' links, two-row links, blocks and
// A_ee^{-1}, every precision the handles hold.
int rank_setup(dd_decomp* D, dd_decomp::Rank& r, cudaStream_t st) {
  const dd_gauge* G = D->op->gauge;
  const dd_clover* C = D->op;
  const SiteMap m = site_map(D, r);
  const int64_t Vh = r.lat.Vh;
  r.gauge.lat = &r.lat;
  r.gauge.prec_mask = G->prec_mask;
  r.gauge.su3_deviation = G->su3_deviation;
  for (int pi = 0; pi < 3; ++pi) {
    if (!G->links[pi].ptr) continue;
    const int ng = groups36(pi);
    DD_TRY(r.gauge.links[pi].alloc((size_t)2 * ng * Vh * 16));
    for (int p = 0; p < 2; ++p)
      DD_TRY(dom_copy<uint4>(m, p, G->U(pi, p), reinterpret_cast<char*>(r.gauge.links[pi].ptr) + (size_t)p * ng * Vh * 16,
                             ng, 1, 1, st));
  }
  // the two-row copies (domains read three rows when the parent holds the
  // eight-real FP32 form)
  if (G->recon32 == 12 && G->links32r.ptr) {
    const int ng = G->recon_groups();
    DD_TRY(r.gauge.links32r.alloc((size_t)2 * ng * Vh * 16));
    for (int p = 0; p < 2; ++p)
      DD_TRY(dom_copy<uint4>(m, p, G->U2(p), reinterpret_cast<char*>(r.gauge.links32r.ptr) + (size_t)p * ng * Vh * 16,
                             ng, 1, 1, st));
    r.gauge.recon32 = G->recon32;
  }
  if (G->recon16 && G->links16r.ptr) {
    DD_TRY(r.gauge.links16r.alloc((size_t)2 * 6 * Vh * 16));
    for (int p = 0; p < 2; ++p)
      DD_TRY(dom_copy<uint4>(m, p, G->U2h(p), reinterpret_cast<char*>(r.gauge.links16r.ptr) + (size_t)p * 6 * Vh * 16,
                             6, 1, 1, st));
    r.gauge.recon16 = G->recon16;
  }
  r.clov.gauge = &r.gauge;
  r.clov.lat = &r.lat;
  r.clov.m0 = C->m0;
  r.clov.csw = C->csw;
  r.clov.prec_mask = C->prec_mask;
  for (int pi = 0; pi < 3; ++pi) {
    if (!C->clov[pi].ptr) continue;
    const int ng = groups36(pi);
    DD_TRY(r.clov.clov[pi].alloc((size_t)2 * ng * Vh * 16));
    for (int p = 0; p < 2; ++p)
      DD_TRY(dom_copy<uint4>(m, p, C->M(pi, p), reinterpret_cast<char*>(r.clov.clov[pi].ptr) + (size_t)p * ng * Vh * 16,
                             ng, 1, 1, st));
    if (C->ainv[pi].ptr) {
      // A_ee^{-1}: the even sites only, ng groups per site
      DD_TRY(r.clov.ainv[pi].alloc((size_t)ng * Vh * 16));
      DD_TRY(dom_copy<uint4>(m, 0, C->Ainv(pi), r.clov.ainv[pi].ptr, ng, 1, 1, st));
    }
  }
  // boundary sites: a hop crosses a split seam
  std::vector<int> b[2];
  const int* n = r.lat.dims;
  for (int t = 0; t < n[0]; ++t)
    for (int z = 0; z < n[1]; ++z)
      for (int y = 0; y < n[2]; ++y)
        for (int x = 0; x < n[3]; ++x) {
          const int c[4] = {t, z, y, x};
          bool cross = false;
          for (int mu = 0; mu < 4; ++mu)
            if (D->grid[mu] > 1 && (c[mu] == 0 || c[mu] == n[mu] - 1)) cross = true;
          if (!cross) continue;
          const int p = (t + z + y + x) & 1;
          const int lex = ((t * n[1] + z) * n[2] + y) * n[3] + x;
          b[p].push_back(p * (int)Vh + (lex >> 1));
        }
  r.nb[0] = (int64_t)b[0].size();
  r.nb[1] = (int64_t)b[1].size();
  std::vector<int> all(b[0]);
  all.insert(all.end(), b[1].begin(), b[1].end());
  if (!all.empty()) {
    DD_TRY(r.bsites.alloc(all.size() * sizeof(int)));
    DD_CUDA(cudaMemcpyAsync(r.bsites.ptr, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    DD_CUDA(cudaStreamSynchronize(st));
  }
  return DD_OK;
}

int rank_index(const int grid[4], const int c[4]) { return ((c[0] * grid[1] + c[1]) * grid[2] + c[2]) * grid[3] + c[3]; }

// The half field of parity p of a native buffer holding a full field (subset
// 0) or one parity (subset 1: odd, 2: even) of `lat`.
char* half_ptr(const dd_lattice* lat, int prec, int subset, void* base, int nrhs, int p) {
  const size_t hb = field_bytes(lat, prec, 1, nrhs);
  char* b = reinterpret_cast<char*>(base);
  if (subset == 0) return b + (size_t)p * hb;
  return b;
}

int copy_field(dd_decomp* D, dd_decomp::Rank& r, int prec, int subset, void* global, int nrhs, int to_local,
               DevBuf& local, cudaStream_t st) {
  const SiteMap m = site_map(D, r);
  for (int p = 0; p < 2; ++p) {
    if (subset == 1 && p == 0) continue;
    if (subset == 2 && p == 1) continue;
    char* g = half_ptr(D->op->lat, prec, subset, global, nrhs, p);
    char* l = reinterpret_cast<char*>(local.ptr) + (size_t)p * field_bytes(&r.lat, prec, 1, nrhs);
    const int G = spinor_groups(prec);
    DD_TRY(dom_copy<uint4>(m, p, to_local ? g : l, to_local ? l : g, G, nrhs, to_local, st));
    if (prec == P16) {  // the site scales after the components
      char* gs = g + (size_t)D->op->lat->Vh * nrhs * 3 * 16;
      char* ls = l + (size_t)r.lat.Vh * nrhs * 3 * 16;
      DD_TRY(dom_copy<float>(m, p, to_local ? gs : ls, to_local ? ls : gs, 1, nrhs, to_local, st));
    }
  }
  return DD_OK;
}

HalfField half_of(const dd_lattice* lat, int prec, DevBuf& buf, int nrhs, int p) {
  Field f = field_view(lat, prec, 0, buf.ptr, nrhs);
  return f.h[p];
}

// Arguments of one rank's stencil launch with the local handles.
DomHopArgs rank_args(dd_decomp* D, dd_decomp::Rank& r, int prec, int nrhs) {
  DomHopArgs A;
  std::memset(&A, 0, sizeof(A));
  HopArgs& a = A.h;
  a.g = r.lat.geom();
  a.nrhs = nrhs;
  a.gstride = r.lat.Vh * nrhs;
  const int pi = prec_index(prec);
  for (int p = 0; p < 2; ++p) {
    a.U[p] = r.gauge.U(pi, p);
    a.M[p] = r.clov.M(pi, p);
  }
  a.recon = prec == P32 && nrhs == 1 ? r.gauge.recon32 : prec == P16 && nrhs == 1 && r.gauge.recon16 ? 12 : 0;
  if (a.recon) {
    a.U[0] = prec == P32 ? r.gauge.U2(0) : r.gauge.U2h(0);
    a.U[1] = prec == P32 ? r.gauge.U2(1) : r.gauge.U2h(1);
  }
  a.rhs_block = 1;
  for (int mu = 0; mu < 4; ++mu) {
    A.d.off[mu] = r.off[mu];
    A.d.N[mu] = D->op->lat->dims[mu];
    A.d.xch[mu] = D->grid[mu] > 1;
    int64_t nf = 1;
    for (int k = 0; k < 4; ++k)
      if (k != mu) nf *= r.lat.dims[k];
    A.d.nface[mu] = nf;
    A.f.lam_send[mu] = r.buf(mu, 0);
    A.f.chi_send[mu] = r.buf(mu, 1);
    A.f.lam_recv[mu] = r.buf(mu, 2);
    A.f.chi_recv[mu] = r.buf(mu, 3);
  }
  A.bsites = reinterpret_cast<const int*>(r.bsites.ptr);
  A.nb[0] = r.nb[0];
  A.nb[1] = r.nb[1];
  return A;
}

cudaError_t pack(int prec, const DomHopArgs& A, bool dag, cudaStream_t st) {
  if (prec == P64) return launch_face_pack<P64, P64>(A, dag, st);
  if (prec == P32) return launch_face_pack<P32, P32>(A, dag, st);
  return launch_face_pack<P16, P16>(A, dag, st);
}

cudaError_t hop(int prec, const DomHopArgs& A, bool dag, int epi, bool boundary, cudaStream_t st) {
  if (prec == P64) return launch_hop_dd<P64, P64, P64>(A, dag, epi, boundary, st);
  if (prec == P32) return launch_hop_dd<P32, P32, P32>(A, dag, epi, boundary, st);
  return launch_hop_dd<P16, P16, P16>(A, dag, epi, boundary, st);
}

// One decomposed stencil launch over all ranks (Algorithm 3): pack the seams,
// send them (copies on the communication stream), run the interior sites,
// wait for the messages, run the boundary sites.
int round_trip(dd_decomp* D, int prec, std::vector<DomHopArgs>& A, bool dag, int epi, cudaStream_t st) {
  const int n = (int)D->ranks.size();
  for (int i = 0; i < n; ++i) {
    const cudaError_t e = pack(prec, A[i], dag, st);
    if (e != cudaSuccess) return cuda_fail(e, "face pack");
  }
  DD_CUDA(cudaEventRecord(D->ev_pack, st));
  DD_CUDA(cudaStreamWaitEvent(D->comm, D->ev_pack, 0));
  for (int i = 0; i < n; ++i) {
    dd_decomp::Rank& r = *D->ranks[i];
    for (int mu = 0; mu < 4; ++mu) {
      if (D->grid[mu] < 2) continue;
      // lambda goes to the rank at -mu, chi to the rank at +mu
      DD_CUDA(cudaMemcpyAsync(D->ranks[r.lo[mu]]->buf(mu, 2), r.buf(mu, 0), r.msg[mu], cudaMemcpyDeviceToDevice,
                              D->comm));
      DD_CUDA(cudaMemcpyAsync(D->ranks[r.hi[mu]]->buf(mu, 3), r.buf(mu, 1), r.msg[mu], cudaMemcpyDeviceToDevice,
                              D->comm));
    }
  }
  DD_CUDA(cudaEventRecord(D->ev_comm, D->comm));
  for (int i = 0; i < n; ++i) {
    const cudaError_t e = hop(prec, A[i], dag, epi, false, st);
    if (e != cudaSuccess) return cuda_fail(e, "interior stencil");
  }
  DD_CUDA(cudaStreamWaitEvent(st, D->ev_comm, 0));
  for (int i = 0; i < n; ++i) {
    const cudaError_t e = hop(prec, A[i], dag, epi, true, st);
    if (e != cudaSuccess) return cuda_fail(e, "boundary stencil");
  }
  return DD_OK;
}

int check_fields(dd_decomp* D, int prec, int nrhs) {
  if (D->field_prec != prec || D->field_nrhs != nrhs)
    return fail(DD_ERR_ARG, "rank fields hold another precision or RHS count: scatter first");
  return DD_OK;
}

}  // namespace

extern "C" {

int dd_decomp_create(const dd_clover* op, const int grid[4], dd_decomp** out) {
  if (!op || !grid || !out) return fail(DD_ERR_ARG, "null argument");
  std::unique_ptr<dd_decomp> D(new (std::nothrow) dd_decomp);
  if (!D) return fail(DD_ERR_OOM, "host allocation failed");
  D->op = op;
  int nr = 1;
  for (int mu = 0; mu < 4; ++mu) {
    const int n = op->lat->dims[mu];
    if (grid[mu] < 1 || n % grid[mu] != 0 || (n / grid[mu]) % 2 != 0)
      return fail(DD_ERR_ARG, "every extent must split into grid[mu] local extents that are even and >= 2");
    D->grid[mu] = grid[mu];
    D->local[mu] = n / grid[mu];
    nr *= grid[mu];
  }
  if (nr < 1 || nr > 4096) return fail(DD_ERR_ARG, "1 to 4096 ranks");
  DD_CUDA(cudaStreamCreateWithFlags(&D->comm, cudaStreamNonBlocking));
  DD_CUDA(cudaEventCreateWithFlags(&D->ev_pack, cudaEventDisableTiming));
  DD_CUDA(cudaEventCreateWithFlags(&D->ev_comm, cudaEventDisableTiming));
  for (int i = 0; i < nr; ++i) {
    std::unique_ptr<dd_decomp::Rank> r(new (std::nothrow) dd_decomp::Rank);
    if (!r) return fail(DD_ERR_OOM, "host allocation failed");
    int c[4], rem = i;
    for (int mu = 3; mu >= 0; --mu) {
      c[mu] = rem % grid[mu];
      rem /= grid[mu];
    }
    for (int mu = 0; mu < 4; ++mu) {
      r->coord[mu] = c[mu];
      r->off[mu] = c[mu] * D->local[mu];
      r->lat.dims[mu] = D->local[mu];
      int cl[4] = {c[0], c[1], c[2], c[3]}, ch[4] = {c[0], c[1], c[2], c[3]};
      cl[mu] = (c[mu] + grid[mu] - 1) % grid[mu];
      ch[mu] = (c[mu] + 1) % grid[mu];
      r->lo[mu] = rank_index(grid, cl);
      r->hi[mu] = rank_index(grid, ch);
    }
    r->lat.t_bc = op->lat->t_bc;
    r->lat.V = (int64_t)D->local[0] * D->local[1] * D->local[2] * D->local[3];
    r->lat.Vh = r->lat.V / 2;
    DD_TRY(rank_setup(D.get(), *r, 0));
    D->ranks.push_back(std::move(r));
  }
  DD_CUDA(cudaDeviceSynchronize());
  *out = D.release();
  return DD_OK;
}

int dd_decomp_destroy(dd_decomp* D) {
  delete D;
  return DD_OK;
}

int dd_decomp_info(const dd_decomp* D, int rank, int* coord4, int* offset4, int* local4, int64_t* boundary_sites) {
  if (!D || rank < 0 || rank >= (int)D->ranks.size()) return fail(DD_ERR_ARG, "bad handle or rank");
  const dd_decomp::Rank& r = *D->ranks[rank];
  for (int mu = 0; mu < 4; ++mu) {
    if (coord4) coord4[mu] = r.coord[mu];
    if (offset4) offset4[mu] = r.off[mu];
    if (local4) local4[mu] = r.lat.dims[mu];
  }
  if (boundary_sites) *boundary_sites = r.nb[0] + r.nb[1];
  return (int)D->ranks.size();
}

int dd_decomp_scatter(dd_decomp* D, int prec, int subset, const void* global, int nrhs, void* stream) {
  if (!D || !global || nrhs < 1) return fail(DD_ERR_ARG, "null argument or nrhs < 1");
  if (prec != P64 && prec != P32 && prec != P16) return fail(DD_ERR_ARG, "bad precision");
  if (subset != 0 && subset != 1) return fail(DD_ERR_ARG, "subset must be 0 (full) or 1 (odd sites)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (auto& r : D->ranks) {
    const size_t fb = field_bytes(&r->lat, prec, 0, nrhs);
    DD_TRY(r->fin.ensure(fb));
    DD_TRY(r->fout.ensure(fb));
    DD_TRY(r->ftmp.ensure(fb));
    DD_TRY(copy_field(D, *r, prec, subset, const_cast<void*>(global), nrhs, 1, r->fin, st));
  }
  D->field_prec = prec;
  D->field_nrhs = nrhs;
  return DD_OK;
}

int dd_decomp_gather(dd_decomp* D, int prec, int subset, void* global, int nrhs, void* stream) {
  if (!D || !global || nrhs < 1) return fail(DD_ERR_ARG, "null argument or nrhs < 1");
  if (subset != 0 && subset != 1) return fail(DD_ERR_ARG, "subset must be 0 (full) or 1 (odd sites)");
  DD_TRY(check_fields(D, prec, nrhs));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (auto& r : D->ranks) DD_TRY(copy_field(D, *r, prec, subset, global, nrhs, 0, r->fout, st));
  return DD_OK;
}

int dd_decomp_apply(dd_decomp* D, int which, int prec, int nrhs, void* stream) {
  if (!D) return fail(DD_ERR_ARG, "null handle");
  if (which != DD_OP_D && which != DD_OP_DH && which != DD_OP_DHAT && which != DD_OP_DHAT_H)
    return fail(DD_ERR_ARG, "operator must be D, D^H, Dhat or Dhat^H");
  DD_TRY(check_fields(D, prec, nrhs));
  const int pi = prec_index(prec);
  if (!D->op->gauge->links[pi].ptr || !D->op->clov[pi].ptr)
    return fail(DD_ERR_UNSUPPORTED, "precision not created in the gauge/operator handles");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool dag = which == DD_OP_DH || which == DD_OP_DHAT_H;
  std::vector<DomHopArgs> A;
  for (auto& rp : D->ranks) {
    dd_decomp::Rank& r = *rp;
    size_t total = 0;
    for (int mu = 0; mu < 4; ++mu) {
      int64_t nf = 1;
      for (int k = 0; k < 4; ++k)
        if (k != mu) nf *= r.lat.dims[k];
      r.msg[mu] = D->grid[mu] < 2 ? 0
                  : prec == P64  ? face_msg_bytes<double>(nf, nrhs, false)
                                 : face_msg_bytes<float>(nf, nrhs, prec == P16);
      r.msg[mu] = (r.msg[mu] + 255) / 256 * 256;
      total += 4 * r.msg[mu];
    }
    DD_TRY(r.faces.ensure(total > 0 ? total : 256));
    A.push_back(rank_args(D, r, prec, nrhs));
  }
  const int n = (int)D->ranks.size();
  if (which == DD_OP_D || which == DD_OP_DH) {
    for (int i = 0; i < n; ++i) {
      dd_decomp::Rank& r = *D->ranks[i];
      HopArgs& a = A[i].h;
      a.npar = 2;
      a.p0 = 0;
      a.beta = -0.5;
      for (int p = 0; p < 2; ++p) {
        a.in[p] = half_of(&r.lat, prec, r.fin, nrhs, p);
        a.y[p] = a.in[p];
        a.out[p] = half_of(&r.lat, prec, r.fout, nrhs, p);
      }
    }
    return round_trip(D, prec, A, dag, EPI_D, st);
  }
  // Dhat = A_oo - D_oe A_ee^{-1} D_eo on the odd halves: tmp_e = A_ee^{-1}
  // (1/2 H_eo in_o), then out_o = A_oo in_o - 1/2 H_oe tmp_e
  std::vector<DomHopArgs> B = A;
  for (int i = 0; i < n; ++i) {
    dd_decomp::Rank& r = *D->ranks[i];
    HopArgs& a = A[i].h;
    a.npar = 1;
    a.p0 = 0;
    a.in[1] = half_of(&r.lat, prec, r.fin, nrhs, 1);
    a.out[0] = half_of(&r.lat, prec, r.ftmp, nrhs, 0);
    a.M[0] = r.clov.Ainv(pi);
    a.beta = 0.5;
    HopArgs& b = B[i].h;
    b.npar = 1;
    b.p0 = 1;
    b.in[0] = half_of(&r.lat, prec, r.ftmp, nrhs, 0);
    b.y[1] = half_of(&r.lat, prec, r.fin, nrhs, 1);
    b.out[1] = half_of(&r.lat, prec, r.fout, nrhs, 1);
    b.beta = -0.5;
  }
  DD_TRY(round_trip(D, prec, A, dag, EPI_AINV, st));
  return round_trip(D, prec, B, dag, EPI_D, st);
}

int dd_decomp_dot(dd_decomp* D, int prec, int subset, int nrhs, double* dots_host, void* stream) {
  if (!D || !dots_host) return fail(DD_ERR_ARG, "null argument");
  if (prec != P64 && prec != P32) return fail(DD_ERR_ARG, "dots of FP64 or FP32 fields");
  if (subset != 0 && subset != 1) return fail(DD_ERR_ARG, "subset must be 0 (full) or 1 (odd sites)");
  DD_TRY(check_fields(D, prec, nrhs));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  DevBuf partials, out;
  DD_TRY(partials.alloc((size_t)blas_partials_len(nrhs) * sizeof(double2)));
  DD_TRY(out.alloc((size_t)nrhs * sizeof(double2)));
  // each rank's partial inner products over its own sites, then the sum over
  // ranks in rank order (the allreduce of the Arnoldi dots)
  for (size_t i = 0; i < D->ranks.size(); ++i) {
    dd_decomp::Rank& r = *D->ranks[i];
    const size_t hb = field_bytes(&r.lat, prec, 1, nrhs);
    const size_t o = subset == 1 ? hb : 0;
    const int64_t L = (int64_t)((subset == 1 ? hb : 2 * hb) / 16);
    VecList vs;
    vs.p[0] = reinterpret_cast<const char*>(r.fout.ptr) + o;
    const void* w = reinterpret_cast<const char*>(r.fin.ptr) + o;
    const int add = i == 0 ? 0 : 1;
    if (prec == P64)
      DD_TRY(blas_multidot<P64>(vs, 1, w, L, nrhs, (double2*)out.ptr, add, (double2*)partials.ptr, st));
    else
      DD_TRY(blas_multidot<P32>(vs, 1, w, L, nrhs, (double2*)out.ptr, add, (double2*)partials.ptr, st));
  }
  DD_CUDA(cudaMemcpyAsync(dots_host, out.ptr, (size_t)nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
  DD_CUDA(cudaStreamSynchronize(st));
  return DD_OK;
}

}  // extern "C"

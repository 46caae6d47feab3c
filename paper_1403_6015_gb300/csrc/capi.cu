// C ABI of the GB300 HODLR library (declared in include/hodlr.h): argument checks, the tree
// of index ranges, device allocation, and the order of the kernel launches for build,
// factor, solve, log det and log-likelihood.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "ff.cuh"
#include "hodlr_internal.cuh"

using hodlr::Ctx;

namespace {

hodlr_status fail(Ctx* c, hodlr_status s, const std::string& msg) {
  if (c) c->last_error = msg;
  return s;
}

hodlr_status cuda_fail(Ctx* c, cudaError_t e, const char* where) {
  cudaGetLastError();
  return fail(c, e == cudaErrorMemoryAllocation ? HODLR_ENOMEM : HODLR_ECUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define TRY_CUDA(c, expr, where)                         \
  do {                                                   \
    cudaError_t _e = (expr);                             \
    if (_e != cudaSuccess) return cuda_fail(c, _e, where); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t dalloc(T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) return cudaSuccess;
  return cudaMalloc((void**)p, sizeof(T) * (size_t)count);
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

int kappa_for(int64_t n, int leaf) {
  int k = 0;
  while (((int64_t)leaf << k) < n) ++k;
  return k;
}

__global__ void k_check_finite(const double* x, int64_t m, int32_t* flag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m && !isfinite(x[i])) atomicOr(flag, 1);
}

void free_factor_buffers(Ctx* c) {
  dfree(c->phi); dfree(c->pan); dfree(c->part); dfree(c->part2); dfree(c->half); dfree(c->Z);
  dfree(c->cnt);
  dfree(c->rank_dev);
  c->R_cap = 0;
}

void free_all(Ctx* c) {
  free_factor_buffers(c);
  dfree(c->nodes); dfree(c->xs); dfree(c->perm);
  dfree(c->item_node); dfree(c->item_start); dfree(c->wide_nodes); dfree(c->wide_cross); dfree(c->node_witem0); dfree(c->node_witem1); dfree(c->node_item0); dfree(c->node_item1); dfree(c->raw);
  dfree(c->cheb_q); dfree(c->cheb_coef);
  dfree(c->st_rank); dfree(c->st_row); dfree(c->st_col); dfree(c->st_done); dfree(c->st_ok);
  dfree(c->st_zero); dfree(c->st_phase); dfree(c->st_nused); dfree(c->st_used);
  dfree(c->st_delta); dfree(c->st_s2); dfree(c->aca_part); dfree(c->active);
  dfree(c->Y); dfree(c->ysort); dfree(c->leafL); dfree(c->leaf_logdet); dfree(c->node_logdet); dfree(c->leaf_perm);
  dfree(c->scal); dfree(c->dflags); dfree(c->tmpvec); dfree(c->ry); dfree(c->rw); dfree(c->exp_tab); dfree(c->xrel); dfree(c->Mlu); dfree(c->Mpiv);
  dfree(c->big_i32); dfree(c->big_slots); dfree(c->big_perm); dfree(c->split_buf);
  dfree(c->hyp);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  dfree(c->sweep_idx);
  if (c->batch_args) cudaFree(c->batch_args);
  c->batch_args = nullptr;
  c->batch_cap = 0;
  c->batch_first_cap = 0;
  dfree(c->batch_first);
  dfree(c->boxes);
  dfree(c->feat);
  if (c->h_active) cudaFreeHost(c->h_active);
  c->h_active = nullptr;
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
}

// Tree of index ranges (Sec. 3): node (j, k) has id 2^j - 1 + k, left child gets the first
// floor(m/2) points. Begins in [0, 2^(kappa+1)), sizes in [2^(kappa+1), 2^(kappa+2)).
void build_tree(Ctx* c) {
  int64_t tot = (int64_t)2 << c->kappa;
  c->h_nodes.assign((size_t)(2 * tot), 0);
  int32_t* nb = c->h_nodes.data();
  int32_t* ns = nb + tot;
  nb[0] = 0;
  ns[0] = (int32_t)c->n;
  for (int64_t id = 0; id < ((int64_t)1 << c->kappa) - 1; ++id) {
    int32_t m = ns[id], ml = m / 2;
    nb[2 * id + 1] = nb[id];
    ns[2 * id + 1] = ml;
    nb[2 * id + 2] = nb[id] + ml;
    ns[2 * id + 2] = m - ml;
  }
  int mx = 0;
  for (int64_t k = 0; k < ((int64_t)1 << c->kappa); ++k)
    mx = std::max(mx, ns[((int64_t)1 << c->kappa) - 1 + k]);
  c->max_leaf_size = mx;
}

hodlr_status setup_aca(Ctx* c) {
  int K = c->kappa;
  int nint = (1 << K) - 1;
  if (nint == 0) return HODLR_OK;
  const int32_t* nb = c->h_nodes.data();
  const int32_t* ns = nb + ((int64_t)2 << K);
  // work items: first the kAcaTile-row tiles of the nodes with a child above kSmallNode
  // points (one block each), node id owning items [i0[id], i1[id]); then, for the nodes
  // whose rank cap exceeds kWideRank, kWideTile-row tiles [wi0[id], wi1[id]) too, which take
  // over from the 1024-row tiles once the node's rank reaches kWideRank; then one item per
  // small node (one warp each)
  std::vector<int32_t> inode, istart, i0(nint + 1), i1(nint + 1, 0), wide;
  std::vector<int32_t> wi0(nint + 1, -1), wi1(nint + 1, -1);
  for (int pass = 0; pass < 3; ++pass) {
    if (pass == 1) c->n_big_items = (int64_t)inode.size();
    if (pass == 2) c->n_wide_items = (int64_t)inode.size() - c->n_big_items;
    for (int id = 0; id < nint; ++id) {
      int32_t m = std::max(ns[2 * id + 1], ns[2 * id + 2]);
      bool small = m <= hodlr::kSmallNode;
      bool wd = !small && std::min(std::min(ns[2 * id + 1], ns[2 * id + 2]), c->max_rank) > hodlr::kWideRank;
      if ((pass == 0 && small) || (pass == 1 && !wd) || (pass == 2 && !small)) continue;
      if (pass == 1) wide.push_back(id);
      const int tile = pass == 1 ? hodlr::kWideTile : hodlr::kAcaTile;
      (pass == 1 ? wi0 : i0)[id] = (int32_t)inode.size();
      for (int32_t s = 0; s < m || s == 0; s += tile) {
        inode.push_back(id);
        istart.push_back(s);
        if (small) break;
      }
      (pass == 1 ? wi1 : i1)[id] = (int32_t)inode.size();
    }
  }
  c->n_wide_nodes = (int)wide.size();
  i0[nint] = i1[nint] = (int32_t)inode.size();
  c->n_items = (int64_t)inode.size();
  c->h_raw_off.assign(K, 0);
  c->h_rcap.assign(K, 0);
  int64_t off = 0;
  for (int j = 0; j < K; ++j) {
    int64_t half = (c->n + ((int64_t)2 << j) - 1) >> (j + 1);
    c->h_rcap[j] = (int)std::min<int64_t>(c->max_rank, half);
    c->h_raw_off[j] = off;
    off += c->n * c->h_rcap[j];
  }
  c->raw_elems = off;
  int us = 2 * c->max_rank + 2;
  TRY_CUDA(c, dalloc(&c->item_node, c->n_items), "alloc items");
  TRY_CUDA(c, dalloc(&c->item_start, c->n_items), "alloc items");
  TRY_CUDA(c, dalloc(&c->node_item0, nint + 1), "alloc items");
  TRY_CUDA(c, dalloc(&c->node_item1, nint + 1), "alloc items");
  TRY_CUDA(c, dalloc(&c->raw, c->raw_elems), "alloc raw panel");
  TRY_CUDA(c, dalloc(&c->st_rank, nint), "alloc aca state");
  TRY_CUDA(c, dalloc(&c->st_row, nint), "alloc aca state");
  TRY_CUDA(c, dalloc(&c->st_col, nint), "alloc aca state");
  TRY_CUDA(c, dalloc(&c->st_done, nint), "alloc aca state");
  TRY_CUDA(c, dalloc(&c->st_ok, nint), "alloc aca state");
  TRY_CUDA(c, dalloc(&c->st_zero, nint), "alloc aca state");
  TRY_CUDA(c, dalloc(&c->st_phase, nint), "alloc aca state");
  TRY_CUDA(c, dalloc(&c->st_nused, nint), "alloc aca state");
  TRY_CUDA(c, dalloc(&c->st_used, (int64_t)nint * us), "alloc aca state");
  TRY_CUDA(c, dalloc(&c->st_delta, nint), "alloc aca state");
  TRY_CUDA(c, dalloc(&c->st_s2, nint), "alloc aca state");
  TRY_CUDA(c, dalloc(&c->aca_part, c->n_items * (4 + 2 * c->max_rank)), "alloc aca partials");
  TRY_CUDA(c, dalloc(&c->wide_nodes, (int64_t)wide.size()), "alloc items");
  TRY_CUDA(c, dalloc(&c->node_witem0, nint + 1), "alloc items");
  TRY_CUDA(c, dalloc(&c->node_witem1, nint + 1), "alloc items");
  TRY_CUDA(c, dalloc(&c->wide_cross, (int64_t)wide.size() * ((c->max_rank + 127) / 128)), "alloc items");
  if (!wide.empty())
    TRY_CUDA(c, cudaMemcpyAsync(c->wide_nodes, wide.data(), 4 * wide.size(), cudaMemcpyHostToDevice, c->stream), "upload");
  if (c->compression == 1) {
    TRY_CUDA(c, dalloc(&c->cheb_q, nint), "alloc chebyshev state");
    TRY_CUDA(c, dalloc(&c->cheb_coef, (int64_t)hodlr::cheb_coef_elems(nint)), "alloc chebyshev state");
  }
  TRY_CUDA(c, cudaMemcpyAsync(c->item_node, inode.data(), 4 * inode.size(), cudaMemcpyHostToDevice, c->stream), "upload");
  TRY_CUDA(c, cudaMemcpyAsync(c->item_start, istart.data(), 4 * istart.size(), cudaMemcpyHostToDevice, c->stream), "upload");
  TRY_CUDA(c, cudaMemcpyAsync(c->node_item0, i0.data(), 4 * i0.size(), cudaMemcpyHostToDevice, c->stream), "upload");
  TRY_CUDA(c, cudaMemcpyAsync(c->node_item1, i1.data(), 4 * i1.size(), cudaMemcpyHostToDevice, c->stream), "upload");
  TRY_CUDA(c, cudaMemcpyAsync(c->node_witem0, wi0.data(), 4 * wi0.size(), cudaMemcpyHostToDevice, c->stream), "upload");
  TRY_CUDA(c, cudaMemcpyAsync(c->node_witem1, wi1.data(), 4 * wi1.size(), cudaMemcpyHostToDevice, c->stream), "upload");
  TRY_CUDA(c, cudaStreamSynchronize(c->stream), "upload");
  ++c->syncs;
  return HODLR_OK;
}

// Buffers whose sizes depend on the per-level ranks h_rl (set before the call).
hodlr_status size_buffers(Ctx* c) {
  int K = c->kappa;
  int nint = (1 << K) - 1;
  c->h_coff.assign(K + 1, 0);
  for (int j = 0; j < K; ++j) c->h_coff[j + 1] = c->h_coff[j] + c->h_rl[j];
  c->R = c->h_coff[K];
  int64_t nleaf = (int64_t)1 << K;
  // per-leaf partials of level j (r_j x (c_j + r_j + max_nrhs) each) for the levels whose
  // half sums are segmented sums: the finest, and those below a sweep step not in product
  // form; the others get their half sums directly (2^(j+1) r_j w_j values)
  int64_t pstride = 1, direct_el = 0;
  bool big = false;
  for (int j = 0; j < K; ++j) {
    const int64_t rw = (int64_t)c->h_rl[j] * (c->h_coff[j] + c->h_rl[j] + c->max_nrhs);
    if (j + 1 < K && hodlr::gemm_step(*c, j + 1)) direct_el = std::max(direct_el, rw << (j + 1));
    else pstride = std::max(pstride, rw);
    big |= c->h_rl[j] > hodlr::kSmemRank;  // a blocked node step (levels_big.cu)
  }
  pstride = std::max<int64_t>(pstride, c->R);  // the matvec stores R partials per leaf
  int64_t zel = 1, hel = 1, mlu = 0, piv = 0;
  c->h_mlu_off.assign(K, 0);
  c->h_piv_off.assign(K, 0);
  for (int j = 0; j < K; ++j) {
    int r = c->h_rl[j];
    zel = std::max<int64_t>(zel, ((int64_t)1 << j) * 2 * r * (c->h_coff[j] + c->max_nrhs));
    zel = std::max<int64_t>(zel, ((int64_t)2 << j) * c->R);
    c->h_mlu_off[j] = mlu;
    c->h_piv_off[j] = piv;
    mlu += ((int64_t)1 << j) * 4 * r * r;
    piv += ((int64_t)1 << j) * 2 * r;
    hel += ((int64_t)2 << j) * r;
  }
  hel = std::max<int64_t>(hel, (nleaf + 1) * pstride);
  hel = std::max<int64_t>(hel, direct_el);
  // the fused sweep's last block of a level-j half sums 2^(K-j-1) partials of r_j w_j values
  c->fused_work = 0;
  for (int j = 0; j < K; ++j)
    c->fused_work = std::max<int64_t>(c->fused_work, ((int64_t)1 << (K - j - 1)) *
                                      c->h_rl[j] * (c->h_coff[j] + c->h_rl[j] + c->max_nrhs));
  bool realloc = c->R_cap < c->R || !c->part || c->part_stride < pstride || c->z_elems < zel ||
                 c->half_elems < hel;
  if (realloc) {
    free_factor_buffers(c);
    int64_t Rc = std::max<int64_t>(c->R, 1);
    TRY_CUDA(c, dalloc(&c->phi, c->n * Rc), "alloc panels");
    TRY_CUDA(c, dalloc(&c->pan, c->n * Rc), "alloc panels");
    TRY_CUDA(c, dalloc(&c->part, nleaf * pstride), "alloc partials");
    TRY_CUDA(c, dalloc(&c->part2, std::max<int64_t>(nleaf / 64 + 1, 8) * pstride + 4096), "alloc partials");
    TRY_CUDA(c, dalloc(&c->half, hel), "alloc partials");
    TRY_CUDA(c, dalloc(&c->Z, 2 * zel), "alloc Z");
    TRY_CUDA(c, dalloc(&c->cnt, nleaf + nleaf / 2 + 2), "alloc counters");
    TRY_CUDA(c, dalloc(&c->rank_dev, std::max(nint, 1)), "alloc ranks");
    c->R_cap = Rc;
    c->part_stride = pstride;
    c->z_elems = zel;
    c->half_elems = hel;
  }
  if (big) {
    // blocked node steps: per node sign and barrier counter, published panel candidates,
    // the substitution's row orders (2 r_j per node of the largest level)
    TRY_CUDA(c, hodlr::big_setup(*c), "large-rank setup");
    int64_t perm_el = 1;
    for (int j = 0; j < K; ++j) perm_el = std::max<int64_t>(perm_el, ((int64_t)2 << j) * c->h_rl[j]);
    if (!c->big_i32) {
      c->big_nodes = std::max<int64_t>(nleaf / 2, 1);
      TRY_CUDA(c, dalloc(&c->big_i32, 2 * c->big_nodes), "alloc large-rank scratch");
      TRY_CUDA(c, dalloc(&c->big_slots, hodlr::big_slot_elems(c->coop_cap)), "alloc large-rank scratch");
    }
    // split-K partial half sums: every width the sweep steps in product form can use
    // (factor mode with 1 .. max_nrhs right-hand sides, solve mode)
    int64_t split_el = 0;
    for (int u = 1; u < K; ++u) {
      if (!hodlr::gemm_step(*c, u)) continue;
      for (int nr = 1; nr <= c->max_nrhs; ++nr)
        for (int w : {c->h_coff[u] + nr, nr}) {
          const int S = hodlr::half_sum_splits(*c, u, w);
          if (S > 1) split_el = std::max<int64_t>(split_el, ((int64_t)S << u) * c->h_rl[u - 1] * w);
        }
    }
    if (c->split_cap < split_el) {
      dfree(c->split_buf);
      TRY_CUDA(c, dalloc(&c->split_buf, split_el), "alloc split sums");
      c->split_cap = split_el;
    }
    if (c->big_perm_cap < perm_el) {
      dfree(c->big_perm);
      TRY_CUDA(c, dalloc(&c->big_perm, perm_el), "alloc large-rank scratch");
      c->big_perm_cap = perm_el;
    }
  }
  if (c->mlu_cap < mlu || c->piv_cap < piv) {
    dfree(c->Mlu);
    dfree(c->Mpiv);
    TRY_CUDA(c, dalloc(&c->Mlu, std::max<int64_t>(mlu, 1)), "alloc node LU");
    TRY_CUDA(c, dalloc(&c->Mpiv, std::max<int64_t>(piv, 1)), "alloc node LU");
    c->mlu_cap = std::max<int64_t>(mlu, 1);
    c->piv_cap = std::max<int64_t>(piv, 1);
  }
  return HODLR_OK;
}

bool capturing(Ctx* c) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c->stream, &st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return st != cudaStreamCaptureStatusNone;
}

// Compression of all off-diagonal blocks, then the rank-padded compact panels. Adaptive
// mode reads the ranks back (one synchronisation); presized mode uses the fixed level
// ranks and leaves any violation in the device flags.
hodlr_status compress(Ctx* c) {
  int K = c->kappa;
  int nint = (1 << K) - 1;
  c->compressed = false;
  c->factored = false;
  c->rank_capped = false;
  bool cap = capturing(c);
  if (!cap) cudaEventRecord(c->ev[2], c->stream);
  int steps = 0;
  if (c->compression == 1)
    TRY_CUDA(c, hodlr::launch_cheb(*c), "chebyshev compression");
  else
    TRY_CUDA(c, hodlr::launch_aca(*c, &steps), "aca");
  if (!c->presized) {
    c->h_rank.assign(nint, 0);
    std::vector<int32_t> ok(nint, 1);
    if (nint > 0) {
      TRY_CUDA(c, cudaMemcpyAsync(c->h_rank.data(), c->st_rank, 4 * (size_t)nint, cudaMemcpyDeviceToHost, c->stream), "ranks");
      TRY_CUDA(c, cudaMemcpyAsync(ok.data(), c->st_ok, 4 * (size_t)nint, cudaMemcpyDeviceToHost, c->stream), "ranks");
      TRY_CUDA(c, cudaStreamSynchronize(c->stream), "ranks");
      ++c->syncs;
    }
    for (int id = 0; id < nint; ++id)
      if (!ok[id]) c->rank_capped = true;
    c->h_rl.assign(K, 0);
    for (int j = 0; j < K; ++j) {
      int mx = 0;
      for (int k = 0; k < (1 << j); ++k) mx = std::max(mx, c->h_rank[(1 << j) - 1 + k]);
      c->h_rl[j] = mx;
    }
    hodlr_status s = size_buffers(c);
    if (s != HODLR_OK) return s;
  }
  // the panels keep their own copy of the ranks
  if (nint > 0)
    TRY_CUDA(c, cudaMemcpyAsync(c->rank_dev, c->st_rank, 4 * (size_t)nint, cudaMemcpyDeviceToDevice, c->stream), "ranks");
  TRY_CUDA(c, hodlr::launch_pack(*c), "pack");
  if (!cap) cudaEventRecord(c->ev[3], c->stream);
  c->compressed = true;
  return HODLR_OK;
}

}  // namespace

extern "C" {

void hodlr_default_opts(hodlr_opts* o) {
  if (!o) return;
  o->precision = 0;
  o->rank_mode = 0;
  o->max_rank = hodlr::kDefaultMaxRank;
  o->max_nrhs = 16;
  o->refine_tol = 1e-10;
  o->refine_maxit = 0;
  o->stream = nullptr;
  o->rq_alpha = 1.0;
  o->compression = 0;
}

const char* hodlr_status_string(hodlr_status s) {
  switch (s) {
    case HODLR_OK: return "OK";
    case HODLR_EINVAL: return "EINVAL";
    case HODLR_ENOMEM: return "ENOMEM";
    case HODLR_ENOTSPD: return "ENOTSPD";
    case HODLR_ERANK: return "ERANK";
    case HODLR_ETIMEOUT: return "ETIMEOUT";
    case HODLR_ESTATE: return "ESTATE";
    case HODLR_ECUDA: return "ECUDA";
  }
  return "UNKNOWN";
}

const char* hodlr_last_error(const hodlr_ctx* ctx) {
  const Ctx* c = reinterpret_cast<const Ctx*>(ctx);
  return c ? c->last_error.c_str() : "null context";
}

void hodlr_destroy(hodlr_ctx* ctx) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_all(c);
  delete c;
}

static bool bad_theta(const double* th) {
  return !th || !std::isfinite(th[0]) || !std::isfinite(th[1]) || !(th[0] > 0) || !(th[1] > 0);
}

hodlr_status hodlr_build(const double* x, int64_t n, int d, hodlr_kernel kernel,
                         const double* theta, double sigma2, int leaf, double eps,
                         const hodlr_opts* o, hodlr_ctx** out) {
  if (!out) return HODLR_EINVAL;
  *out = nullptr;
  hodlr_opts opts;
  hodlr_default_opts(&opts);
  if (o) opts = *o;
  if (!x || n < 1 || n >= ((int64_t)1 << 31) || d < 1 || d > hodlr::kMaxDim || leaf < 1 ||
      leaf > hodlr::kMaxLeaf || !(eps > 0) || !std::isfinite(eps) || !(sigma2 >= 0) ||
      !std::isfinite(sigma2) || bad_theta(theta) || (int)kernel < 0 ||
      (int)kernel > HODLR_K_BIHARMONIC ||
      (kernel == HODLR_K_RQ && (!(opts.rq_alpha > 0) || !std::isfinite(opts.rq_alpha))) ||
      (hodlr::kind_indefinite(kernel) && opts.precision != 0) ||
      (opts.compression != 0 && opts.compression != 1) || (opts.compression == 1 && d != 1) ||
      opts.max_rank < 1 || opts.max_rank > hodlr::kMaxRank || opts.max_nrhs < 1 ||
      (opts.precision != 0 && opts.precision != 1) || opts.refine_maxit < 0 ||
      (opts.refine_maxit > 0 && (!(opts.refine_tol > 0) || !std::isfinite(opts.refine_tol))))
    return HODLR_EINVAL;
  Ctx* c = new (std::nothrow) Ctx;
  if (!c) return HODLR_ENOMEM;
  c->n = n;
  c->d = d;
  c->kind = (int)kernel;
  c->alpha = opts.rq_alpha;
  c->compression = opts.compression;
  c->indefinite = hodlr::kind_indefinite(kernel);
  c->ell = theta[0];
  c->amp = theta[1];
  c->sigma2 = sigma2;
  c->eps = eps;
  c->leaf = leaf;
  c->max_rank = opts.max_rank;
  c->max_nrhs = opts.max_nrhs;
  c->precision = opts.precision;
  c->refine_tol = opts.refine_tol;
  c->refine_maxit = opts.refine_maxit;
  if (const char* e = std::getenv("HODLR_LEAF_THREADS")) c->leaf_threads = std::atoi(e);
  if (const char* e = std::getenv("HODLR_LEAF_THREADS64")) c->leaf_threads64 = std::atoi(e);
  if (const char* e = std::getenv("HODLR_LEAF_TC")) c->leaf_tc = std::atoi(e) != 0;
  if (const char* e = std::getenv("HODLR_NO_FUSED")) c->no_fused = std::atoi(e) != 0;
  c->stream = (cudaStream_t)opts.stream;
  c->kappa = kappa_for(n, leaf);
  auto bail = [&](hodlr_status s) {
    free_all(c);
    delete c;
    return s;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) return bail(HODLR_ECUDA);
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  for (auto& e : c->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return bail(HODLR_ECUDA);
  build_tree(c);
  int64_t tot = (int64_t)2 << c->kappa;
  int64_t nleaf = (int64_t)1 << c->kappa;
  if (dalloc(&c->nodes, 2 * tot) || dalloc(&c->xs, n * d) || dalloc(&c->perm, n) ||
      dalloc(&c->dflags, 4) || dalloc(&c->scal, 8) || dalloc(&c->active, 1) ||
      dalloc(&c->hyp, hodlr::kHypLen) || dalloc(&c->exp_tab, 64) ||
      dalloc(&c->Y, n * c->max_nrhs) || dalloc(&c->ysort, n) || dalloc(&c->tmpvec, n * c->max_nrhs) ||
      dalloc(&c->leaf_logdet, nleaf) || dalloc(&c->node_logdet, std::max<int64_t>(nleaf - 1, 1)) ||
      dalloc(&c->leafL, nleaf * hodlr::kMaxLeaf * hodlr::kMaxLeaf) ||
      (c->indefinite && dalloc(&c->leaf_perm, nleaf * hodlr::kMaxLeaf)) ||
      (c->refine_maxit > 0 && (dalloc(&c->ry, n * c->max_nrhs) ||
                               dalloc(&c->rw, hodlr::refine_work_elems(n)))) ||
      cudaMallocHost(&c->h_active, sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    return bail(HODLR_ENOMEM);
  }
  cudaMemcpyAsync(c->nodes, c->h_nodes.data(), 4 * c->h_nodes.size(), cudaMemcpyHostToDevice, c->stream);
  if (hodlr::launch_exp_table(*c) != cudaSuccess) return bail(HODLR_ECUDA);
  // points on the device (row-major n x d), finiteness check
  const double* xd = x;
  double* xtmp = nullptr;
  if (!is_device_ptr(x)) {
    if (dalloc(&xtmp, n * d) != cudaSuccess) return bail(HODLR_ENOMEM);
    cudaMemcpyAsync(xtmp, x, sizeof(double) * n * d, cudaMemcpyHostToDevice, c->stream);
    xd = xtmp;
  }
  cudaMemsetAsync(c->dflags, 0, 4, c->stream);
  k_check_finite<<<(unsigned)((n * d + 255) / 256), 256, 0, c->stream>>>(xd, n * d, c->dflags);
  ++c->launches;
  int32_t fl = 0;
  cudaMemcpyAsync(&fl, c->dflags, 4, cudaMemcpyDeviceToHost, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    dfree(xtmp);
    return bail(HODLR_ECUDA);
  }
  if (fl) {
    dfree(xtmp);
    return bail(HODLR_EINVAL);
  }
  cudaEventRecord(c->ev[0], c->stream);
  cudaError_t e = d == 1 ? hodlr::launch_sort_1d(*c, xd) : hodlr::launch_sort_kd(*c, xd);
  cudaEventRecord(c->ev[1], c->stream);
  cudaStreamSynchronize(c->stream);
  dfree(xtmp);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bail(e == cudaErrorMemoryAllocation ? HODLR_ENOMEM : HODLR_ECUDA);
  }
  hodlr_status s = setup_aca(c);
  if (s != HODLR_OK) return bail(s);
  if (c->precision == 1 && c->kappa > 0) {
    if (dalloc(&c->xrel, (int64_t)c->kappa * d * n) != cudaSuccess) return bail(HODLR_ENOMEM);
    if (hodlr::launch_xrel(*c) != cudaSuccess) return bail(HODLR_ECUDA);
  }
  if (hodlr::launch_set_hyp(*c, c->ell, c->amp, c->sigma2) != cudaSuccess) return bail(HODLR_ECUDA);
  s = compress(c);
  if (s != HODLR_OK) return bail(s);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(HODLR_ECUDA);
  cudaEventElapsedTime(&c->phase_ms[0], c->ev[0], c->ev[1]);
  cudaEventElapsedTime(&c->phase_ms[1], c->ev[2], c->ev[3]);
  *out = reinterpret_cast<hodlr_ctx*>(c);
  if (c->rank_capped) {
    c->last_error = "compression reached max_rank before eps (Chebyshev: needed more than 64 nodes) in at least one block";
    return HODLR_ERANK;
  }
  return HODLR_OK;
}

hodlr_status hodlr_rebuild(hodlr_ctx* ctx, const double* theta, double sigma2) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return HODLR_EINVAL;
  if (bad_theta(theta) || !(sigma2 >= 0) || !std::isfinite(sigma2))
    return fail(c, HODLR_EINVAL, "rebuild: bad theta or sigma2");
  c->ell = theta[0];
  c->amp = theta[1];
  c->sigma2 = sigma2;
  TRY_CUDA(c, hodlr::launch_set_hyp(*c, c->ell, c->amp, c->sigma2), "hyperparameters");
  hodlr_status s = compress(c);
  if (s != HODLR_OK) return s;
  if (c->presized) return HODLR_OK;  // stream-ordered; violations go to the device flags
  TRY_CUDA(c, cudaStreamSynchronize(c->stream), "rebuild");
  ++c->syncs;
  cudaEventElapsedTime(&c->phase_ms[1], c->ev[2], c->ev[3]);
  if (c->rank_capped) return fail(c, HODLR_ERANK, "compression reached max_rank before eps (Chebyshev: needed more than 64 nodes) in at least one block");
  return HODLR_OK;
}

// Stage a (possibly host) n x nrhs column-major input; returns a device pointer and its ld.
static hodlr_status stage_in(Ctx* c, const double* y, int nrhs, int64_t ld, const double** yd,
                             int64_t* ldd) {
  if (is_device_ptr(y)) {
    *yd = y;
    *ldd = ld;
    return HODLR_OK;
  }
  TRY_CUDA(c, cudaMemcpy2DAsync(c->tmpvec, sizeof(double) * c->n, y, sizeof(double) * ld,
                                sizeof(double) * c->n, nrhs, cudaMemcpyHostToDevice, c->stream),
           "copy y");
  *yd = c->tmpvec;
  *ldd = c->n;
  return HODLR_OK;
}

static hodlr_status write_out(Ctx* c, double* x, int nrhs, int64_t ld) {
  if (is_device_ptr(x)) {
    TRY_CUDA(c, hodlr::launch_scatter_rhs(*c, x, ld, nrhs), "scatter");
    return HODLR_OK;
  }
  TRY_CUDA(c, hodlr::launch_scatter_rhs(*c, c->tmpvec, c->n, nrhs), "scatter");
  TRY_CUDA(c, cudaMemcpy2DAsync(x, sizeof(double) * ld, c->tmpvec, sizeof(double) * c->n,
                                sizeof(double) * c->n, nrhs, cudaMemcpyDeviceToHost, c->stream),
           "copy x");
  TRY_CUDA(c, cudaStreamSynchronize(c->stream), "copy x");
  ++c->syncs;
  return HODLR_OK;
}

static hodlr_status check_flags(Ctx* c) {
  int32_t fl = 0;
  TRY_CUDA(c, cudaMemcpyAsync(&fl, c->dflags, 4, cudaMemcpyDeviceToHost, c->stream), "flags");
  TRY_CUDA(c, cudaStreamSynchronize(c->stream), "flags");
  ++c->syncs;
  if (fl & hodlr::kFlagTimeout) {
    c->factored = false;
    return fail(c, HODLR_ETIMEOUT, "a bounded device wait (grid barrier of a large-rank LU panel) gave up");
  }
  if (fl & hodlr::kFlagNotSpd) {
    c->factored = false;
    return fail(c, HODLR_ENOTSPD, c->indefinite ? "a leaf pivot or node determinant was zero"
                                                : "a leaf pivot or node determinant was not positive");
  }
  c->det_sign = (fl & hodlr::kFlagNegDet) ? -1 : 1;
  return HODLR_OK;
}

// Level sweep: one launch per level when each level's reductions are small enough for
// one block per half-node, else the segmented three-launch path.
static cudaError_t sweep(Ctx* c, int nrhs, bool factor_mode) {
  int rmax = 0;
  for (int r : c->h_rl) rmax = std::max(rmax, r);
  if (c->fused_work <= ((int64_t)1 << 22) && !c->no_fused && rmax <= hodlr::kSmemRank)
    return hodlr::launch_levels_fused(*c, nrhs, factor_mode);
  return hodlr::launch_levels(*c, nrhs, factor_mode);
}

// Right-hand sides into c->Y in tree order (and, with refinement on, their copy in c->ry).
static cudaError_t gather_rhs(Ctx* c, const double* y, int64_t ld, int nrhs) {
  cudaError_t e = hodlr::launch_gather_rhs(*c, y, ld, nrhs);
  if (e == cudaSuccess && c->refine_maxit > 0)
    e = cudaMemcpyAsync(c->ry, c->Y, sizeof(double) * c->n * nrhs, cudaMemcpyDeviceToDevice, c->stream);
  return e;
}

// Iterative refinement of the nrhs solutions in c->Y (not in the paper): per column,
// r = y - C~ x with the FP64 HODLR product, stop when ||r|| / ||y|| <= refine_tol, else
// solve C d = r with the stored factor (in place in the work vector) and x += d, at most
// refine_maxit times. Under stream capture, and in the sweep and batched forms (fixed =
// true, so that their eager first evaluation matches the replays), there is no host check:
// exactly refine_maxit corrections per column.
static hodlr_status refine(Ctx* c, int nrhs, bool fixed = false) {
  c->refine_corr = 0;
  c->refine_res = 0.0;
  if (c->refine_maxit <= 0) return HODLR_OK;
  bool cap = fixed || capturing(c);
  int64_t n = c->n;
  double* r = c->rw;
  double* part = c->rw + n;
  double* ratio = c->rw + hodlr::refine_work_elems(n) - 8;
  for (int col = 0; col < nrhs; ++col) {
    double* x = c->Y + (int64_t)col * n;
    const double* y = c->ry + (int64_t)col * n;
    for (int it = 0; it <= c->refine_maxit; ++it) {
      if (cap && it == c->refine_maxit) break;
      TRY_CUDA(c, hodlr::launch_matvec(*c, x, r), "refine: matvec");
      TRY_CUDA(c, hodlr::launch_residual(*c, y, r, part, ratio), "refine: residual");
      if (!cap) {
        double res = 0.0;
        TRY_CUDA(c, cudaMemcpyAsync(&res, ratio, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "refine");
        TRY_CUDA(c, cudaStreamSynchronize(c->stream), "refine");
        ++c->syncs;
        if (res <= c->refine_tol || it == c->refine_maxit) {
          c->refine_res = std::max(c->refine_res, res);
          break;
        }
      }
      double* ysave = c->Y;
      c->Y = r;
      cudaError_t e = c->precision == 1 ? hodlr::launch_leaf_solve_ff(*c, 1) : hodlr::launch_leaf_solve(*c, 1);
      if (e == cudaSuccess) e = sweep(c, 1, false);
      c->Y = ysave;
      TRY_CUDA(c, e, "refine: correction solve");
      TRY_CUDA(c, hodlr::launch_axpy(*c, x, r), "refine: update");
      ++c->refine_corr;
    }
  }
  return HODLR_OK;
}

// Factor with nrhs right-hand sides already gathered into c->Y (nrhs may be 0).
static hodlr_status factor_impl(Ctx* c, int nrhs) {
  if (!c->compressed) return fail(c, HODLR_ESTATE, "not compressed");
  if (c->factored) return fail(c, HODLR_ESTATE, "already factored (rebuild first)");
  c->solve_timed = false;
  bool cap = capturing(c);
  if (!cap) cudaEventRecord(c->ev[4], c->stream);
  // the leaf stage reads the original U/V from phi and writes the working panel (every
  // column, every point), so no copy of phi is needed first
  if (!c->presized) TRY_CUDA(c, cudaMemsetAsync(c->dflags, 0, 4, c->stream), "flags");
  if (!cap) cudaEventRecord(c->ev[6], c->stream);
  if (c->precision == 1)
    TRY_CUDA(c, hodlr::launch_leaf_factor_ff(*c, nrhs), "leaf factor (double-float)");
  else
    TRY_CUDA(c, hodlr::launch_leaf_factor(*c, nrhs), "leaf factor");
  if (!cap) cudaEventRecord(c->ev[7], c->stream);
  TRY_CUDA(c, sweep(c, nrhs, true), "levels");
  TRY_CUDA(c, hodlr::launch_logdet_sum(*c), "logdet");
  if (!cap) cudaEventRecord(c->ev[5], c->stream);
  c->factored = true;
  c->nrhs_fused = nrhs;
  if (c->presized) return HODLR_OK;  // no synchronisation: see hodlr_status_flags
  hodlr_status s = check_flags(c);
  cudaEventElapsedTime(&c->phase_ms[2], c->ev[4], c->ev[5]);
  cudaEventElapsedTime(&c->phase_ms[4], c->ev[6], c->ev[7]);
  cudaEventElapsedTime(&c->phase_ms[5], c->ev[7], c->ev[5]);
  return s;
}

hodlr_status hodlr_factor(hodlr_ctx* ctx) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return HODLR_EINVAL;
  return factor_impl(c, 0);
}

hodlr_status hodlr_factor_solve(hodlr_ctx* ctx, const double* y, double* x, int nrhs,
                                int64_t ld) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return HODLR_EINVAL;
  if (!y || !x || nrhs < 1 || nrhs > c->max_nrhs || ld < c->n)
    return fail(c, HODLR_EINVAL, "factor_solve: bad y/x/nrhs/ld");
  if (c->factored) return fail(c, HODLR_ESTATE, "already factored (rebuild first)");
  const double* yd = nullptr;
  int64_t ldd = 0;
  hodlr_status s = stage_in(c, y, nrhs, ld, &yd, &ldd);
  if (s != HODLR_OK) return s;
  TRY_CUDA(c, gather_rhs(c, yd, ldd, nrhs), "gather");
  s = factor_impl(c, nrhs);
  if (s != HODLR_OK) return s;
  s = refine(c, nrhs);
  if (s != HODLR_OK) return s;
  return write_out(c, x, nrhs, ld);
}

hodlr_status hodlr_solve(hodlr_ctx* ctx, const double* y, double* x, int nrhs, int64_t ld) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return HODLR_EINVAL;
  if (!c->factored) return fail(c, HODLR_ESTATE, "solve before factor");
  if (!y || !x || nrhs < 1 || ld < c->n) return fail(c, HODLR_EINVAL, "solve: bad y/x/nrhs/ld");
  for (int c0 = 0; c0 < nrhs; c0 += c->max_nrhs) {
    int nb = std::min(c->max_nrhs, nrhs - c0);
    const double* yd = nullptr;
    int64_t ldd = 0;
    hodlr_status s = stage_in(c, y + (int64_t)c0 * ld, nb, ld, &yd, &ldd);
    if (s != HODLR_OK) return s;
    cudaEventRecord(c->ev[4], c->stream);
    TRY_CUDA(c, gather_rhs(c, yd, ldd, nb), "gather");
    if (c->precision == 1)
      TRY_CUDA(c, hodlr::launch_leaf_solve_ff(*c, nb), "leaf solve (double-float)");
    else
      TRY_CUDA(c, hodlr::launch_leaf_solve(*c, nb), "leaf solve");
    TRY_CUDA(c, sweep(c, nb, false), "levels");
    s = refine(c, nb);
    if (s != HODLR_OK) return s;
    cudaEventRecord(c->ev[5], c->stream);
    c->solve_timed = true;
    s = write_out(c, x + (int64_t)c0 * ld, nb, ld);
    if (s != HODLR_OK) return s;
  }
  return HODLR_OK;
}

static hodlr_status write_scalar(Ctx* c, const double* src, double* out) {
  if (is_device_ptr(out)) {
    TRY_CUDA(c, cudaMemcpyAsync(out, src, sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "out");
    return HODLR_OK;
  }
  TRY_CUDA(c, cudaMemcpyAsync(out, src, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "out");
  TRY_CUDA(c, cudaStreamSynchronize(c->stream), "out");
  ++c->syncs;
  return HODLR_OK;
}

hodlr_status hodlr_logdet(hodlr_ctx* ctx, double* logdet) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !logdet) return HODLR_EINVAL;
  if (!c->factored) return fail(c, HODLR_ESTATE, "logdet before factor");
  return write_scalar(c, c->scal, logdet);
}

hodlr_status hodlr_logdet_signed(hodlr_ctx* ctx, double* logabsdet, int* sign) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !logabsdet || !sign) return HODLR_EINVAL;
  if (!c->factored) return fail(c, HODLR_ESTATE, "logdet before factor");
  *sign = c->det_sign;
  return write_scalar(c, c->scal, logabsdet);
}

hodlr_status hodlr_loglik(hodlr_ctx* ctx, const double* y, double* out) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !y || !out) return HODLR_EINVAL;
  if (c->indefinite) return fail(c, HODLR_EINVAL, "loglik: the kernel's C is indefinite (not a covariance)");
  const double* yd = nullptr;
  int64_t ldd = 0;
  hodlr_status s = stage_in(c, y, 1, c->n, &yd, &ldd);
  if (s != HODLR_OK) return s;
  TRY_CUDA(c, gather_rhs(c, yd, ldd, 1), "gather");
  if (!c->factored) {
    s = factor_impl(c, 1);
    if (s != HODLR_OK) return s;
  } else {
    if (c->precision == 1)
      TRY_CUDA(c, hodlr::launch_leaf_solve_ff(*c, 1), "leaf solve (double-float)");
    else
      TRY_CUDA(c, hodlr::launch_leaf_solve(*c, 1), "leaf solve");
    TRY_CUDA(c, sweep(c, 1, false), "levels");
  }
  s = refine(c, 1);
  if (s != HODLR_OK) return s;
  TRY_CUDA(c, hodlr::launch_quad_loglik(*c), "loglik");
  return write_scalar(c, c->scal + 2, out);
}

hodlr_status hodlr_presize(hodlr_ctx* ctx, const int32_t* level_ranks, int nlevels) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return HODLR_EINVAL;
  if (c->indefinite && level_ranks)
    return fail(c, HODLR_EINVAL, "presize: not for an indefinite kernel (its sign needs a read-back)");
  if (c->compression == 1 && level_ranks)
    return fail(c, HODLR_EINVAL, "presize: not with Chebyshev compression");
  if (!level_ranks) {
    c->presized = false;
    c->graph_valid = false;
    return HODLR_OK;
  }
  if (nlevels != c->kappa) return fail(c, HODLR_EINVAL, "presize: nlevels must equal kappa");
  for (int j = 0; j < nlevels; ++j)
    if (level_ranks[j] < 0 || level_ranks[j] + 1 > c->max_rank)
      return fail(c, HODLR_EINVAL, "presize: level rank outside [0, max_rank - 1]");
  c->h_rl.assign(level_ranks, level_ranks + nlevels);
  hodlr_status s = size_buffers(c);
  if (s != HODLR_OK) return s;
  c->presized = true;
  c->graph_valid = false;
  c->compressed = false;
  c->factored = false;
  TRY_CUDA(c, cudaMemsetAsync(c->dflags, 0, 4, c->stream), "flags");
  return HODLR_OK;
}

hodlr_status hodlr_status_flags(hodlr_ctx* ctx, int32_t* flags) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !flags) return HODLR_EINVAL;
  int32_t f = 0;
  TRY_CUDA(c, cudaMemcpyAsync(&f, c->dflags, 4, cudaMemcpyDeviceToHost, c->stream), "flags");
  TRY_CUDA(c, cudaMemsetAsync(c->dflags, 0, 4, c->stream), "flags");
  TRY_CUDA(c, cudaStreamSynchronize(c->stream), "flags");
  ++c->syncs;
  *flags = f;
  return HODLR_OK;
}

// One evaluation for the setting idx[0] of the sweep arrays, ending with out[idx] =
// log-likelihood, status[idx] = device flags of this evaluation, idx += 1.
__global__ void k_store_setting(const double* scal, int32_t* flags, int32_t* idx, double* out,
                                int32_t* status) {
  int b = idx[0];
  out[b] = scal[2];
  if (status) status[b] = flags[0];
  flags[0] = 0;
  idx[0] = b + 1;
}

static hodlr_status sweep_eval(Ctx* c, const double* theta, const double* sigma2, const double* y,
                               double* out, int32_t* status) {
  TRY_CUDA(c, hodlr::launch_load_setting(*c, theta, sigma2, c->sweep_idx), "setting");
  hodlr_status s = compress(c);
  if (s != HODLR_OK) return s;
  TRY_CUDA(c, gather_rhs(c, y, c->n, 1), "gather");
  c->factored = false;
  s = factor_impl(c, 1);
  if (s != HODLR_OK) return s;
  s = refine(c, 1, true);
  if (s != HODLR_OK) return s;
  TRY_CUDA(c, hodlr::launch_quad_loglik(*c), "loglik");
  k_store_setting<<<1, 1, 0, c->stream>>>(c->scal, c->dflags, c->sweep_idx, out, status);
  ++c->launches;
  TRY_CUDA(c, cudaGetLastError(), "store");
  return HODLR_OK;
}

hodlr_status hodlr_loglik_sweep(hodlr_ctx* ctx, int64_t nset, const double* theta,
                                const double* sigma2, const double* y, double* out,
                                int32_t* status) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return HODLR_EINVAL;
  if (!c->presized) return fail(c, HODLR_ESTATE, "sweep: presize the context first");
  if (nset < 1 || !theta || !sigma2 || !y || !out || !is_device_ptr(theta) ||
      !is_device_ptr(sigma2) || !is_device_ptr(y) || !is_device_ptr(out) ||
      (status && !is_device_ptr(status)))
    return fail(c, HODLR_EINVAL, "sweep: device arrays required");
  if (!c->stream) return fail(c, HODLR_EINVAL, "sweep: needs a non-default stream");
  if (!c->sweep_idx) TRY_CUDA(c, dalloc(&c->sweep_idx, 1), "alloc");
  TRY_CUDA(c, cudaMemsetAsync(c->sweep_idx, 0, sizeof(int32_t), c->stream), "sweep");
  bool same = c->graph_valid && c->g_theta == theta && c->g_sigma2 == sigma2 && c->g_y == y &&
              c->g_out == out && c->g_status == status;
  if (!same) {
    // one eager evaluation first (sets kernel attributes), then capture one evaluation
    hodlr_status s = sweep_eval(c, theta, sigma2, y, out, status);
    if (s != HODLR_OK) return s;
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
    cudaGraph_t g = nullptr;
    TRY_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed), "capture");
    int64_t l0 = c->launches;
    s = sweep_eval(c, theta, sigma2, y, out, status);
    c->launches_captured = c->launches - l0;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (s != HODLR_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    TRY_CUDA(c, e, "capture");
    e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    TRY_CUDA(c, e, "instantiate");
    c->graph_valid = true;
    c->g_theta = theta;
    c->g_sigma2 = sigma2;
    c->g_y = y;
    c->g_out = out;
    c->g_status = status;
    c->graph_launches = c->launches_captured;
    nset -= 1;  // the eager evaluation did setting 0
  }
  for (int64_t b = 0; b < nset; ++b) TRY_CUDA(c, cudaGraphLaunch(c->graph_exec, c->stream), "replay");
  c->launches += nset * c->graph_launches;
  return HODLR_OK;
}

hodlr_status hodlr_block_features(hodlr_ctx* ctx, double ell, float* X, int64_t ld) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !X || !(ell > 0) || ld < 12 || !is_device_ptr(X)) return HODLR_EINVAL;
  TRY_CUDA(c, hodlr::launch_block_features(*c, ell, X, ld), "features");
  return HODLR_OK;
}

hodlr_status hodlr_predict_ranks(hodlr_ctx* ctx, hodlr_mlp* mlp, double ell, int margin,
                                 int32_t* level_ranks) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !mlp || !level_ranks || !(ell > 0) || margin < 0) return HODLR_EINVAL;
  int K = c->kappa;
  int nint = (1 << K) - 1;
  if (nint == 0) return HODLR_OK;
  if (!c->feat) TRY_CUDA(c, dalloc(&c->feat, (int64_t)nint * 13), "alloc features");
  float* X = c->feat;
  float* Yp = c->feat + (int64_t)nint * 12;
  TRY_CUDA(c, hodlr::launch_block_features(*c, ell, X, 12), "features");
  TRY_CUDA(c, hodlr::launch_mlp_forward(*c, mlp, X, nint, Yp), "predict");
  std::vector<float> y(nint);
  TRY_CUDA(c, cudaMemcpyAsync(y.data(), Yp, sizeof(float) * nint, cudaMemcpyDeviceToHost, c->stream), "predict");
  TRY_CUDA(c, cudaStreamSynchronize(c->stream), "predict");
  ++c->syncs;
  for (int j = 0; j < K; ++j) {
    int mx = 0;
    for (int k = 0; k < (1 << j); ++k) {
      double r = std::expm1((double)y[(1 << j) - 1 + k]);
      mx = std::max(mx, (int)std::lround(std::max(r, 0.0)));
    }
    level_ranks[j] = std::min(mx + margin, c->max_rank - 1);
  }
  return HODLR_OK;
}

// Lane step r of a batched run: setting b = first + min(r, count - 1) stride into the
// device hyperparameter slot (rounds past count repeat the last setting and store nothing).
__global__ void k_lane_load(double* hyp, int kind, const double* theta, const double* sigma2,
                            const int32_t* round, int64_t first, int64_t stride, int64_t count) {
  int64_t r = round[0];
  int64_t b = first + (r < count ? r : count - 1) * stride;
  double ell = theta[2 * b], amp = theta[2 * b + 1];
  hyp[hodlr::kHypInvEll] = 1.0 / ell;
  hyp[hodlr::kHypAmp] = amp;
  hyp[hodlr::kHypSigma2] = sigma2[b];
  hyp[hodlr::kHypScale] = hodlr::cov_scale(kind, ell);
  hodlr::set_hyp_ff(hyp);
}

__global__ void k_lane_store(const double* scal, int32_t* flags, int32_t* round, double* out,
                             int32_t* status, int64_t first, int64_t stride, int64_t count) {
  int64_t r = round[0];
  if (r < count) {
    int64_t b = first + r * stride;
    out[b] = scal[2];
    if (status) status[b] = flags[0];
  }
  flags[0] = 0;
  round[0] = (int32_t)(r + 1);
}

// A lane's part of a round before the leaf stage: its setting into the hyperparameter
// slot, the compression, the right-hand side.
static hodlr_status lane_pre(const hodlr_batch_lane& L) {
  Ctx* c = reinterpret_cast<Ctx*>(L.ctx);
  k_lane_load<<<1, 1, 0, c->stream>>>(c->hyp, c->kind, L.theta, L.sigma2, c->sweep_idx, L.first,
                                      L.stride, L.count);
  ++c->launches;
  hodlr_status s = compress(c);
  if (s != HODLR_OK) return s;
  TRY_CUDA(c, gather_rhs(c, L.y, c->n, 1), "gather");
  c->factored = false;
  return HODLR_OK;
}

// A lane's part after the leaf stage: level sweep, log det, refinement, log-likelihood,
// and the result into the caller's output.
static hodlr_status lane_post(const hodlr_batch_lane& L) {
  Ctx* c = reinterpret_cast<Ctx*>(L.ctx);
  TRY_CUDA(c, sweep(c, 1, true), "levels");
  TRY_CUDA(c, hodlr::launch_logdet_sum(*c), "logdet");
  c->factored = true;
  c->nrhs_fused = 1;
  hodlr_status s = refine(c, 1, true);
  if (s != HODLR_OK) return s;
  TRY_CUDA(c, hodlr::launch_quad_loglik(*c), "loglik");
  k_lane_store<<<1, 1, 0, c->stream>>>(c->scal, c->dflags, c->sweep_idx, L.out, L.status, L.first,
                                       L.stride, L.count);
  ++c->launches;
  TRY_CUDA(c, cudaGetLastError(), "store");
  return HODLR_OK;
}

// The leaf stage of every lane of one round: per form (FP64, mixed), one persistent
// launch whose CTAs take (lane, leaf) items from a device counter; its argument blocks
// and leaf offsets sit in the first lane's context (written before the rounds).
struct BatchLeaves {
  int nprob[2] = {0, 0};
  int total[2] = {0, 0};
  size_t args_off[2] = {0, 0};  // byte offset of each form's argument blocks in batch_args
  int first_off[2] = {0, 0};    // int offset of each form's offsets in batch_first
  int counter_off = 0;          // two counters after the offsets
};

static hodlr_status plan_leaves(const hodlr_batch_lane* lanes, int nlanes, cudaStream_t origin,
                                BatchLeaves* plan) {
  Ctx* c0 = reinterpret_cast<Ctx*>(lanes[0].ctx);
  const size_t asz[2] = {hodlr::leaf_args_bytes(), hodlr::leaf_args_bytes_ff()};
  std::vector<unsigned char> hargs;
  std::vector<int32_t> hfirst;
  for (int f = 0; f < 2; ++f) {
    plan->args_off[f] = hargs.size();
    plan->first_off[f] = (int)hfirst.size();
    int tot = 0;
    for (int i = 0; i < nlanes; ++i) {
      Ctx* c = reinterpret_cast<Ctx*>(lanes[i].ctx);
      if (c->precision != f) continue;
      size_t at = hargs.size();
      hargs.resize(at + asz[f]);
      if (f == 1) hodlr::leaf_args_fill_ff(*c, 1, hargs.data() + at);
      else hodlr::leaf_args_fill(*c, 1, hargs.data() + at);
      hfirst.push_back(tot);
      tot += 1 << c->kappa;
      ++plan->nprob[f];
    }
    hfirst.push_back(tot);
    plan->total[f] = tot;
  }
  plan->counter_off = (int)hfirst.size();
  hfirst.push_back(0);
  hfirst.push_back(0);
  int64_t need = (int64_t)hargs.size();
  if (need > c0->batch_cap || (int64_t)hfirst.size() > c0->batch_first_cap) {
    if (c0->batch_args) cudaFree(c0->batch_args);
    c0->batch_args = nullptr;
    c0->batch_cap = 0;
    c0->batch_first_cap = 0;
    dfree(c0->batch_first);
    int64_t nf = std::max<int64_t>((int64_t)hfirst.size(), 2 * (int64_t)nlanes + 8);
    if (cudaMalloc(&c0->batch_args, (size_t)std::max<int64_t>(need, 1)) != cudaSuccess ||
        cudaMalloc(&c0->batch_first, sizeof(int32_t) * (size_t)nf) != cudaSuccess) {
      cudaGetLastError();
      return fail(c0, HODLR_ENOMEM, "batched: leaf work list");
    }
    c0->batch_cap = std::max<int64_t>(need, 1);
    c0->batch_first_cap = nf;
  }
  TRY_CUDA(c0, cudaMemcpyAsync(c0->batch_args, hargs.data(), hargs.size(), cudaMemcpyHostToDevice, origin),
           "batched: leaf work list");
  TRY_CUDA(c0, cudaMemcpyAsync(c0->batch_first, hfirst.data(), sizeof(int32_t) * hfirst.size(),
                               cudaMemcpyHostToDevice, origin), "batched: leaf work list");
  return HODLR_OK;
}

static hodlr_status leaves_round(const hodlr_batch_lane* lanes, const BatchLeaves& plan,
                                 cudaStream_t origin) {
  Ctx* c0 = reinterpret_cast<Ctx*>(lanes[0].ctx);
  for (int f = 0; f < 2; ++f) {
    if (plan.nprob[f] == 0) continue;
    int32_t* counter = c0->batch_first + plan.counter_off + f;
    TRY_CUDA(c0, cudaMemsetAsync(counter, 0, sizeof(int32_t), origin), "batched: leaf counter");
    const void* args = static_cast<unsigned char*>(c0->batch_args) + plan.args_off[f];
    const int32_t* first = c0->batch_first + plan.first_off[f];
    cudaError_t e = f == 1 ? hodlr::launch_leaf_factor_multi_ff(args, first, plan.nprob[f], plan.total[f],
                                                                counter, c0->sms, origin)
                           : hodlr::launch_leaf_factor_multi(args, first, plan.nprob[f], plan.total[f],
                                                             counter, c0->sms, origin);
    TRY_CUDA(c0, e, "batched: leaf stage");
    ++c0->launches;
  }
  return HODLR_OK;
}

// One round: every lane's compression and right-hand side on its own stream (fork), the
// persistent leaf launches on the origin stream (join), every lane's sweep and
// log-likelihood on its own stream again (fork), joined into the origin stream.
static hodlr_status batched_round(const hodlr_batch_lane* lanes, int nlanes, cudaStream_t origin,
                                  const BatchLeaves& plan, std::vector<cudaEvent_t>& ev) {
  cudaEventRecord(ev[nlanes], origin);
  for (int i = 0; i < nlanes; ++i) {
    Ctx* c = reinterpret_cast<Ctx*>(lanes[i].ctx);
    cudaStreamWaitEvent(c->stream, ev[nlanes], 0);
    hodlr_status s = lane_pre(lanes[i]);
    if (s != HODLR_OK) return s;
    cudaEventRecord(ev[i], c->stream);
    cudaStreamWaitEvent(origin, ev[i], 0);
  }
  hodlr_status s = leaves_round(lanes, plan, origin);
  if (s != HODLR_OK) return s;
  cudaEventRecord(ev[nlanes + 1], origin);
  for (int i = 0; i < nlanes; ++i) {
    Ctx* c = reinterpret_cast<Ctx*>(lanes[i].ctx);
    cudaStreamWaitEvent(c->stream, ev[nlanes + 1], 0);
    s = lane_post(lanes[i]);
    if (s != HODLR_OK) return s;
    cudaEventRecord(ev[i], c->stream);
    cudaStreamWaitEvent(origin, ev[i], 0);
  }
  return HODLR_OK;
}

hodlr_status hodlr_loglik_batched(const hodlr_batch_lane* lanes, int nlanes, void* stream) {
  if (!lanes || nlanes < 1 || !stream) return HODLR_EINVAL;
  cudaStream_t origin = static_cast<cudaStream_t>(stream);
  int64_t rounds = 0;
  for (int i = 0; i < nlanes; ++i) {
    const hodlr_batch_lane& L = lanes[i];
    Ctx* c = reinterpret_cast<Ctx*>(L.ctx);
    if (!c) return HODLR_EINVAL;
    if (!c->presized) return fail(c, HODLR_EINVAL, "batched: lane context is not presized");
    if (!c->stream || c->stream == origin)
      return fail(c, HODLR_EINVAL, "batched: a lane stream must be non-default and differ from the caller's stream");
    if (L.count < 1 || L.first < 0 || L.stride < 1)
      return fail(c, HODLR_EINVAL, "batched: bad first/stride/count");
    if (!is_device_ptr(L.theta) || !is_device_ptr(L.sigma2) || !is_device_ptr(L.y) ||
        !is_device_ptr(L.out) || (L.status && !is_device_ptr(L.status)))
      return fail(c, HODLR_EINVAL, "batched: theta, sigma2, y, out, status must be device pointers");
    for (int j = 0; j < i; ++j)
      if (lanes[j].ctx == L.ctx) return fail(c, HODLR_EINVAL, "batched: context used by two lanes");
    if (!c->sweep_idx && dalloc(&c->sweep_idx, 1) != cudaSuccess)
      return fail(c, HODLR_ENOMEM, "batched: counter");
    rounds = std::max(rounds, L.count);
  }
  std::vector<cudaEvent_t> ev(nlanes + 2, nullptr);
  for (auto& e : ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (auto& f : ev)
        if (f) cudaEventDestroy(f);
      return HODLR_ECUDA;
    }
  auto cleanup = [&]() {
    for (auto& f : ev)
      if (f) cudaEventDestroy(f);
  };
  // round counters to zero and the leaf work list, ordered before the rounds on origin
  for (int i = 0; i < nlanes; ++i) {
    Ctx* c = reinterpret_cast<Ctx*>(lanes[i].ctx);
    cudaMemsetAsync(c->sweep_idx, 0, sizeof(int32_t), origin);
  }
  BatchLeaves plan;
  hodlr_status ps = plan_leaves(lanes, nlanes, origin, &plan);
  if (ps != HODLR_OK) {
    cleanup();
    return ps;
  }
  // one direct round first (sets kernel attributes outside the capture)
  {
    hodlr_status s = batched_round(lanes, nlanes, origin, plan, ev);
    if (s != HODLR_OK) {
      cleanup();
      return s;
    }
  }
  if (rounds > 1) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed);
    hodlr_status s = HODLR_OK;
    if (e == cudaSuccess) {
      s = batched_round(lanes, nlanes, origin, plan, ev);
      e = cudaStreamEndCapture(origin, &g);
    }
    if (s == HODLR_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    for (int64_t r = 1; r < rounds && s == HODLR_OK && e == cudaSuccess; ++r)
      e = cudaGraphLaunch(ge, origin);
    if (ge) cudaGraphExecDestroy(ge);
    if (s == HODLR_OK && e != cudaSuccess) {
      cudaGetLastError();
      s = fail(reinterpret_cast<Ctx*>(lanes[0].ctx), HODLR_ECUDA,
               std::string("batched: graph capture or replay: ") + cudaGetErrorString(e));
    }
    if (s != HODLR_OK) {
      cleanup();
      return s;
    }
  }
  // events may be destroyed once recorded work is enqueued
  cleanup();
  return HODLR_OK;
}

hodlr_status hodlr_ranks(hodlr_ctx* ctx, int32_t* ranks, int64_t cap, int64_t* count) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return HODLR_EINVAL;
  int64_t m = (int64_t)c->h_rank.size();
  if (count) *count = m;
  if (ranks)
    for (int64_t i = 0; i < m && i < cap; ++i) ranks[i] = c->h_rank[i];
  return HODLR_OK;
}

hodlr_status hodlr_tree(hodlr_ctx* ctx, int* kappa, int64_t* perm) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return HODLR_EINVAL;
  if (kappa) *kappa = c->kappa;
  if (perm) {
    std::vector<int32_t> p(c->n);
    TRY_CUDA(c, cudaMemcpyAsync(p.data(), c->perm, 4 * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream), "perm");
    TRY_CUDA(c, cudaStreamSynchronize(c->stream), "perm");
  ++c->syncs;
    for (int64_t i = 0; i < c->n; ++i) perm[i] = p[i];
  }
  return HODLR_OK;
}

hodlr_status hodlr_matvec(hodlr_ctx* ctx, const double* x, double* y) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !x || !y) return HODLR_EINVAL;
  if (!c->compressed) return fail(c, HODLR_ESTATE, "matvec before build");
  const double* xd = nullptr;
  int64_t ldd = 0;
  hodlr_status s = stage_in(c, x, 1, c->n, &xd, &ldd);
  if (s != HODLR_OK) return s;
  // sorted x into ysort, product into Y[:, 0], then back to caller order
  TRY_CUDA(c, hodlr::launch_gather_rhs(*c, xd, ldd, 1), "gather");
  TRY_CUDA(c, cudaMemcpyAsync(c->ysort, c->Y, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream), "copy");
  TRY_CUDA(c, hodlr::launch_matvec(*c, c->ysort, c->Y), "matvec");
  return write_out(c, y, 1, c->n);
}

static bool valid_tuning(const Ctx* c, const hodlr_tuning* t) {
  if (!t || (t->sweep_mode != 0 && t->sweep_mode != 1)) return false;
  if (t->leaf_kernel != 0 && t->leaf_kernel != 1) return false;
  if (t->sweep_tile < 0 || t->sweep_tile > 6) return false;
  if (c->precision == 1) return t->leaf_threads == 512 || t->leaf_threads == 1024;
  return t->leaf_kernel == 0 &&
         (t->leaf_threads == 256 || t->leaf_threads == 512 || t->leaf_threads == 1024);
}

hodlr_status hodlr_get_tuning(hodlr_ctx* ctx, hodlr_tuning* out) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !out) return HODLR_EINVAL;
  out->leaf_threads = c->precision == 1 ? c->leaf_threads : c->leaf_threads64;
  out->sweep_mode = c->no_fused ? 1 : 0;
  out->leaf_kernel = c->precision == 1 && c->leaf_tc ? 1 : 0;
  out->sweep_tile = c->sweep_tile;
  return HODLR_OK;
}

hodlr_status hodlr_set_tuning(hodlr_ctx* ctx, const hodlr_tuning* t) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return HODLR_EINVAL;
  if (!valid_tuning(c, t))
    return fail(c, HODLR_EINVAL, "set_tuning: leaf_threads, sweep_mode or leaf_kernel");
  if (c->precision == 1) c->leaf_threads = t->leaf_threads;
  else c->leaf_threads64 = t->leaf_threads;
  c->leaf_tc = c->precision == 1 && t->leaf_kernel == 1;
  c->no_fused = t->sweep_mode == 1;
  c->sweep_tile = t->sweep_tile;
  c->graph_valid = false;  // captured graphs hold the old launch shapes
  return HODLR_OK;
}

hodlr_status hodlr_autotune(hodlr_ctx* ctx, const double* y, int reps, hodlr_tuning* best,
                            float* best_ms) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !y || reps < 1 || reps > 100) return HODLR_EINVAL;
  if (!c->compressed) return fail(c, HODLR_ESTATE, "autotune: compress (build or rebuild) first");
  if (capturing(c)) return fail(c, HODLR_ESTATE, "autotune: not under stream capture");
  const double* yd = nullptr;
  int64_t ldd = 0;
  hodlr_status s = stage_in(c, y, 1, c->n, &yd, &ldd);
  if (s != HODLR_OK) return s;
  // candidates: (leaf_threads, leaf_kernel); the tensor-core leaf kernel has one CTA size
  std::vector<std::pair<int, int>> cands =
      c->precision == 1 ? std::vector<std::pair<int, int>>{{512, 0}, {1024, 0}, {512, 1}}
                        : std::vector<std::pair<int, int>>{{256, 0}, {512, 0}, {1024, 0}};
  hodlr_tuning saved;
  hodlr_get_tuning(ctx, &saved);
  hodlr_tuning win = saved;
  float win_ms = -1.0f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return fail(c, HODLR_ECUDA, "autotune: events");
  }
  // sweep configurations: the segmented sweep, then the fused sweep's tile shapes
  std::vector<std::pair<int, int>> sweeps = {{1, 0}, {0, 0}, {0, 1}, {0, 2}, {0, 3}, {0, 4},
                                             {0, 5}, {0, 6}};
  for (const auto& sw : sweeps)
    for (const auto& cand : cands) {
      if (s != HODLR_OK) break;
      hodlr_tuning t{cand.first, sw.first, cand.second, sw.second};
      hodlr_set_tuning(ctx, &t);
      std::vector<float> ms;
      for (int r = 0; r <= reps && s == HODLR_OK; ++r) {
        cudaError_t e = gather_rhs(c, yd, ldd, 1);
        if (e != cudaSuccess) {
          s = fail(c, HODLR_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
          break;
        }
        c->factored = false;
        cudaEventRecord(e0, c->stream);
        s = factor_impl(c, 1);
        cudaEventRecord(e1, c->stream);
        if (s == HODLR_OK && cudaEventSynchronize(e1) == cudaSuccess) {
          float v = 0.0f;
          cudaEventElapsedTime(&v, e0, e1);
          if (r > 0) ms.push_back(v);  // the first run is untimed (attributes, caches)
        }
      }
      if (s != HODLR_OK) break;
      std::sort(ms.begin(), ms.end());
      float med = ms.empty() ? 0.0f : ms[ms.size() / 2];
      if (win_ms < 0.0f || med < win_ms) {
        win_ms = med;
        win = t;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->factored = false;
  if (s != HODLR_OK) {
    hodlr_set_tuning(ctx, &saved);
    return s;
  }
  hodlr_set_tuning(ctx, &win);
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return HODLR_OK;
}

hodlr_status hodlr_predict(hodlr_ctx* ctx, const double* xtest, int64_t m, const double* y,
                           double* mean, double* var) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return HODLR_EINVAL;
  if (!xtest || m < 1 || !y || !mean) return fail(c, HODLR_EINVAL, "predict: bad xtest/m/y/mean");
  if (!c->factored) return fail(c, HODLR_ESTATE, "predict before factor");
  if (capturing(c)) return fail(c, HODLR_ESTATE, "predict: not under stream capture");
  double *xt = nullptr, *alpha = nullptr, *part = nullptr, *res = nullptr;
  auto cleanup = [&]() {
    dfree(xt);
    dfree(alpha);
    dfree(part);
    dfree(res);
  };
  if (dalloc(&xt, m * c->d) || dalloc(&alpha, c->n) ||
      dalloc(&part, hodlr::predict_partial_elems(std::max<int64_t>(m, c->max_nrhs))) ||
      dalloc(&res, 2 * m)) {
    cudaGetLastError();
    cleanup();
    return fail(c, HODLR_ENOMEM, "predict: buffers");
  }
  auto run = [&]() -> hodlr_status {
    TRY_CUDA(c, cudaMemcpyAsync(xt, xtest, sizeof(double) * m * c->d, cudaMemcpyDefault, c->stream), "xtest");
    // alpha = C^-1 y with the stored factor (tree order)
    const double* yd = nullptr;
    int64_t ldd = 0;
    hodlr_status s = stage_in(c, y, 1, c->n, &yd, &ldd);
    if (s != HODLR_OK) return s;
    TRY_CUDA(c, hodlr::launch_gather_rhs(*c, yd, ldd, 1), "gather");
    TRY_CUDA(c, c->precision == 1 ? hodlr::launch_leaf_solve_ff(*c, 1) : hodlr::launch_leaf_solve(*c, 1), "leaf solve");
    TRY_CUDA(c, sweep(c, 1, false), "levels");
    TRY_CUDA(c, cudaMemcpyAsync(alpha, c->Y, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream), "alpha");
    // mean in chunks of test points
    const int64_t chunk = 4096;
    for (int64_t j0 = 0; j0 < m; j0 += chunk) {
      int nc = (int)std::min<int64_t>(chunk, m - j0);
      TRY_CUDA(c, hodlr::launch_cross_dot(*c, xt, j0, nc, alpha, 0, 0, part, 0, res), "mean");
    }
    // variance: k_* columns solved max_nrhs at a time
    if (var) {
      for (int64_t j0 = 0; j0 < m; j0 += c->max_nrhs) {
        int nc = (int)std::min<int64_t>(c->max_nrhs, m - j0);
        TRY_CUDA(c, hodlr::launch_cross_fill(*c, xt, j0, nc), "cross");
        TRY_CUDA(c, c->precision == 1 ? hodlr::launch_leaf_solve_ff(*c, nc) : hodlr::launch_leaf_solve(*c, nc), "leaf solve");
        TRY_CUDA(c, sweep(c, nc, false), "levels");
        TRY_CUDA(c, hodlr::launch_cross_dot(*c, xt, j0, nc, c->Y, c->n, 1, part, 1, res + m), "variance");
      }
    }
    TRY_CUDA(c, cudaMemcpyAsync(mean, res, sizeof(double) * m, cudaMemcpyDefault, c->stream), "mean out");
    if (var)
      TRY_CUDA(c, cudaMemcpyAsync(var, res + m, sizeof(double) * m, cudaMemcpyDefault, c->stream), "var out");
    TRY_CUDA(c, cudaStreamSynchronize(c->stream), "predict");
    ++c->syncs;
    return HODLR_OK;
  };
  hodlr_status s = run();
  cleanup();
  return s;
}

hodlr_status hodlr_refine_info(hodlr_ctx* ctx, int32_t* corrections, double* residual) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return HODLR_EINVAL;
  if (corrections) *corrections = c->refine_corr;
  if (residual) *residual = c->refine_res;
  return HODLR_OK;
}

hodlr_status hodlr_phase_ms(hodlr_ctx* ctx, float* out6) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !out6) return HODLR_EINVAL;
  cudaStreamSynchronize(c->stream);
  if (c->solve_timed) cudaEventElapsedTime(&c->phase_ms[3], c->ev[4], c->ev[5]);
  for (int i = 0; i < 6; ++i) out6[i] = c->phase_ms[i];
  return HODLR_OK;
}

hodlr_status hodlr_counters(hodlr_ctx* ctx, int64_t* out2) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !out2) return HODLR_EINVAL;
  out2[0] = c->launches;
  out2[1] = c->syncs;
  return HODLR_OK;
}

}  // extern "C"

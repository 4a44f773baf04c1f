// api.cpp -- the C ABI of libcopula (see include/copula.h): argument checks,
// the per-call work schedule, the workspace layout and the launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "copula.h"
#include "internal.h"
#include "rankcorr.h"

using namespace cop;

// Gauss-Legendre nodes and weights on [0, 1] (Newton on P_n), n <= 128.
void cop::gauss_legendre01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-15) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * pp * pp);
  }
}

// Spearman's rho = 12 int int C(u,v) du dv - 3 of the Frank (Eq. 10) and
// Gumbel (Eq. 11) copulas on the start-value grids.  Allocates nothing.
void cop::build_start_tables(StartTables& T) {
  constexpr int NG = 96;
  double x[NG], w[NG];
  gauss_legendre01(NG, x, w);
  auto rho = [&](int fam, double th) {
    double s = 0.0;
    for (int i = 0; i < NG; ++i)
      for (int j = 0; j < NG; ++j) {
        const double u = x[i], v = x[j];
        double C;
        if (fam == COPULA_FRANK)
          C = th == 0.0 ? u * v : -std::log1p(std::expm1(-th * u) * std::expm1(-th * v) / std::expm1(-th)) / th;
        else
          C = std::exp(-std::pow(std::pow(-std::log(u), th) + std::pow(-std::log(v), th), 1.0 / th));
        s += w[i] * w[j] * C;
      }
    return 12.0 * s - 3.0;
  };
  for (int j = 0; j < kStartN; ++j) {
    T.frank_rho[j] = (float)rho(COPULA_FRANK, kFrankStart0 + kFrankStartStep * j);
    T.gumbel_rho[j] = (float)rho(COPULA_GUMBEL, kGumbelStart0 + kGumbelStartStep * j);
  }
  // keep the tables strictly increasing for the device-side search
  for (int j = 1; j < kStartN; ++j) {
    if (!(T.frank_rho[j] > T.frank_rho[j - 1])) T.frank_rho[j] = std::nextafter(T.frank_rho[j - 1], 2.0f);
    if (!(T.gumbel_rho[j] > T.gumbel_rho[j - 1])) T.gumbel_rho[j] = std::nextafter(T.gumbel_rho[j - 1], 2.0f);
  }
}


struct copula_ctx {
  int device = 0;
  int sms = 0;
  size_t smem_optin = 0;
  void* staging = nullptr;  // pinned host memory for the per-call schedule
  size_t staging_bytes = 0;
  void* rstage = nullptr;   // pinned host memory for copula_fit_host's results
  size_t rstage_bytes = 0;
  cudaEvent_t staging_done = nullptr;
  bool staging_pending = false;
  StartTables start;
  std::string err;
  bool timing = false;
  bool timed = false;  // the last call recorded the timing events
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaEvent_t sev[kStreamEvents] = {};  // streaming-path stage events
  unsigned long long* stamps = nullptr; // device: the streaming fit kernel's barrier timestamps (timed calls)
  bool stream_timed = false;           // the last timed call ran the streaming path
  int32_t launches = 0;
  // (largest m, threads) per family, from copula_ctx_set_blocks /
  // copula_ctx_set_family_blocks
  std::vector<std::pair<int32_t, int32_t>> blocks[3];
  uint64_t blocks_version = 0;  // bumped whenever a block table changes (invalidates the plan cache)
  int64_t wait_spins = 0;    // streaming grid-barrier poll limit (0: the built-in 2^24)
  int32_t wait_phantom = 0;  // extra arrivals the barriers wait for (tests of the give-up path)
  void* plan_cache = nullptr;  // the last plan and its arguments (PlanCache, below)
  uint64_t next_plan_id = 0;    // ids of cached plans
  uint64_t staging_plan_id = 0; // the cached plan whose upload image the staging holds (0: none)
};

namespace {

int fail(copula_ctx* ctx, int code, const char* what) {
  if (ctx) ctx->err = what;
  return code;
}

int cuda_fail(copula_ctx* ctx, cudaError_t e, const char* where) {
  if (ctx) {
    ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
  }
  return COPULA_ERR_CUDA;
}

copula_opts resolve_opts(const copula_opts* o) {
  copula_opts r;
  copula_opts_default(&r);
  if (o) r = *o;
  if (r.max_iter <= 0) r.max_iter = 64;
  if (!(r.rtol > 0.0)) r.rtol = r.precision == COPULA_PREC_F64 ? 1e-13 : 1e-6;
  return r;
}

int block_for(const copula_ctx* ctx, int m, int family, const copula_opts& o) {
  if (o.block == 0 && ctx && family >= 0 && family < 3) {
    for (const auto& b : ctx->blocks[family])
      if (m <= b.first) return b.second;
  }
  return block_size_for(m, o.block);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// A validated batch: jobs grouped into launch buckets, and the workspace map.
struct Plan {
  uint64_t id = 0;  // nonzero for a context's cached plan (its upload image may still be staged)
  int32_t B = 0;
  int64_t S = 0, n = 0;
  std::vector<Job> jobs;  // LPT order within each bucket, buckets consecutive
  struct Bucket {
    int block, first, count, m_max;
    bool tab_smem;
    size_t smem;
    int grid;                    // CTAs launched
    size_t gws_stride, gws_gs_off;  // per-CTA global scratch (0: none)
  };
  std::vector<Bucket> buckets;
  std::vector<int64_t> dss;  // dataset_subset_start, B+1
  size_t gws_bytes = 0;  // global scratch of the resident launches (buckets run one after another)
  // streaming path: subsets larger than one CTA's shared-memory sort, laid
  // out back to back in compact order
  std::vector<Seg> segs;
  std::vector<Chunk> chunks;
  std::vector<int32_t> bucket_seg;
  int64_t n_stream = 0;
  // workspace offsets
  // [0, off_upload_end): zeroed counters and the schedule, one host copy
  size_t off_counters, off_jobs, off_dss, off_upload_end;
  size_t off_var, off_info, off_status, off_iters, off_gws;
  size_t off_segs = 0, off_chunks = 0, off_bseg = 0, off_spl_key = 0, off_spl_idx = 0, off_bcnt = 0, off_bstart = 0,
         off_mat = 0, off_bof = 0, off_bkey = 0, off_bidx = 0, off_ranku = 0, off_rankv = 0, off_pi = 0,
         off_tab = 0, off_tabv = 0, off_wu = 0, off_wv = 0, off_part = 0, off_state = 0, off_sync = 0;
  int64_t n_mat = 0;  // entries of all chunk x bucket count matrices
  size_t off_end;
};

int ctas_per_sm(const copula_ctx* ctx, int block, size_t smem);
int occupancy_grid(copula_ctx* ctx, int count, int block, size_t smem);

// The last plan a context built and the arguments it was built from: a call
// with the same partition, families, storage type, options and block tables
// reuses it instead of planning again (planning 60,000 subsets takes a few
// milliseconds on the host).
struct PlanCache {
  bool valid = false;
  int32_t dtype = 0, B = 0;
  copula_opts o{};
  uint64_t blocks_version = 0;
  std::vector<int32_t> fam;
  std::vector<int64_t> doff, soff, dss;
  Plan P;
};

int make_plan(copula_ctx* ctx, int32_t dtype, const copula_opts& o, int32_t B, const int32_t* family,
              const int64_t* doff, const int64_t* soff, const int64_t* dss, Plan& P) {
  if (dtype != COPULA_DTYPE_F32 && dtype != COPULA_DTYPE_F64) return fail(ctx, COPULA_ERR_ARG, "bad dtype");
  if (o.precision != COPULA_PREC_F64 && o.precision != COPULA_PREC_F32C) return fail(ctx, COPULA_ERR_ARG, "bad precision");
  if (o.weight < 0 || o.weight > 2) return fail(ctx, COPULA_ERR_ARG, "bad weight");
  if (B < 1 || !doff || !soff || !dss) return fail(ctx, COPULA_ERR_ARG, "missing partition");
  if (doff[0] != 0 || dss[0] != 0) return fail(ctx, COPULA_ERR_ARG, "offsets must start at 0");
  P.B = B;
  P.S = dss[B];
  P.n = doff[B];
  if (P.S < 1 || P.n < 2) return fail(ctx, COPULA_ERR_ARG, "empty input");
  if (soff[0] != 0 || soff[P.S] != P.n) return fail(ctx, COPULA_ERR_ARG, "subset offsets must cover [0, n)");
  const int ks = dtype == COPULA_DTYPE_F32 ? 4 : 8;
  const int rs = o.precision == COPULA_PREC_F32C ? 4 : 8;
  P.dss.assign(dss, dss + B + 1);
  const int64_t res_max = ks == 4 ? COPULA_MAX_SUBSET : COPULA_MAX_SUBSET_F64;
  const int64_t str_max = ks == 4 ? kStreamMax32 : kStreamMax64;
  std::vector<Job> all;
  all.reserve((size_t)P.S);
  P.segs.clear();
  P.chunks.clear();
  P.bucket_seg.clear();
  P.n_stream = 0;
  P.n_mat = 0;
  for (int32_t b = 0; b < B; ++b) {
    const int fam = family ? family[b] : 0;
    if (fam < 0 || fam > 2) return fail(ctx, COPULA_ERR_ARG, "bad family");
    if (dss[b + 1] <= dss[b]) return fail(ctx, COPULA_ERR_ARG, "dataset without subsets");
    if (soff[dss[b]] != doff[b] || soff[dss[b + 1]] != doff[b + 1])
      return fail(ctx, COPULA_ERR_ARG, "subsets do not tile their dataset");
    for (int64_t k = dss[b]; k < dss[b + 1]; ++k) {
      const int64_t m = soff[k + 1] - soff[k];
      if (m < 2) return fail(ctx, COPULA_ERR_ARG, "subset with fewer than 2 rows");
      if (m > str_max) return fail(ctx, COPULA_ERR_UNSUPPORTED, "subset larger than the streaming path fits");
      if (m > res_max) {
        Seg sg;
        sg.off = soff[k];
        sg.c = P.n_stream;
        sg.m = m;
        sg.family = fam;
        sg.subset = (int32_t)k;
        sg.dataset = b;
        sg.pad = 0;
        const int64_t mean = ks == 4 ? kBucketMean32 : kBucketMean64;
        sg.nb = (int32_t)std::max<int64_t>(2, (m + mean - 1) / mean);
        sg.bucket_base = (int32_t)P.bucket_seg.size();
        sg.chunk_first = (int32_t)P.chunks.size();
        for (int64_t c0 = 0; c0 < m; c0 += kChunk)
          P.chunks.push_back(Chunk{(int32_t)P.segs.size(), (int32_t)std::min<int64_t>(kChunk, m - c0), c0});
        sg.chunk_count = (int32_t)P.chunks.size() - sg.chunk_first;
        sg.mat = P.n_mat;
        P.n_mat += (int64_t)sg.chunk_count * sg.nb;
        P.bucket_seg.insert(P.bucket_seg.end(), (size_t)sg.nb, (int32_t)P.segs.size());
        P.segs.push_back(sg);
        P.n_stream += m;
        continue;
      }
      Job j;
      j.off = soff[k];
      j.m = (int32_t)m;
      j.family = fam;
      j.subset = (int32_t)k;
      j.dataset = b;
      j.gs_mode = 0;
      j.pad = 0;
      all.push_back(j);
    }
  }
  // longest subsets first (LPT), grouped by launch block size
  std::stable_sort(all.begin(), all.end(), [](const Job& a, const Job& b) { return a.m > b.m; });
  P.jobs.clear();
  P.buckets.clear();
  for (int blk : {512, 256, 128}) {
    Plan::Bucket bk{blk, (int)P.jobs.size(), 0, 0, false, 0, 0, 0, 0};
    for (const Job& j : all)
      if (block_for(ctx, j.m, j.family, o) == blk) {
        P.jobs.push_back(j);
        bk.m_max = std::max(bk.m_max, j.m);
      }
    bk.count = (int)P.jobs.size() - bk.first;
    if (bk.count == 0) continue;
    const size_t lim = (ctx && ctx->smem_optin) ? std::min(ctx->smem_optin - 2048, kMaxSmem) : kMaxSmem;
    if (res_layout(bk.m_max, ks, rs, false, false, blk).total > lim)
      return fail(ctx, COPULA_ERR_UNSUPPORTED, "subset too large for the shared-memory sort at this dtype");
    // Shared memory first for the tables.  The variance's per-point store
    // goes there too for a subset whose own layout then keeps its CTAs per
    // SM (a rule on m alone, so that the bucket keeps its occupancy and a
    // subset its arithmetic whatever else is in the batch); otherwise FP64
    // keeps it in per-CTA global scratch and FP32 evaluates the terms again.
    bk.tab_smem = res_layout(bk.m_max, ks, rs, true, false, blk).total <= lim;
    int m_gs2 = 0;
    for (int i = bk.first; i < bk.first + bk.count; ++i) {
      Job& j = P.jobs[i];
      const size_t s0 = res_layout(j.m, ks, rs, bk.tab_smem, false, blk).total;
      const size_t s1 = res_layout(j.m, ks, rs, bk.tab_smem, true, blk).total;
      // (without a context, for a size query only: the store is taken as
      // global, so the answer bounds what any context's plan needs)
      const bool gs_smem = ctx && s1 <= lim && ctas_per_sm(ctx, blk, s1) >= ctas_per_sm(ctx, blk, s0);
      j.gs_mode = gs_smem ? 1 : (rs == 8 ? 2 : 0);
      bk.smem = std::max(bk.smem, gs_smem ? s1 : s0);
      if (j.gs_mode == 2) m_gs2 = std::max(m_gs2, j.m);
    }
    bk.grid = (ctx && ctx->sms > 0) ? occupancy_grid(ctx, bk.count, blk, bk.smem) : bk.count;
    bk.gws_gs_off = bk.tab_smem ? 0 : align256(2 * (size_t)bk.m_max * rs);
    const size_t per_cta = bk.gws_gs_off + (m_gs2 > 0 ? var_store_entries(m_gs2, blk, rs) * rs : 0);
    bk.gws_stride = align256(per_cta);
    P.gws_bytes = std::max(P.gws_bytes, (size_t)bk.grid * bk.gws_stride);
    P.buckets.push_back(bk);
  }
  size_t o2 = 0;
  P.off_counters = o2; o2 = align256(o2 + (kJobCounters + (size_t)B) * sizeof(int32_t));
  P.off_jobs = o2; o2 = align256(o2 + P.jobs.size() * sizeof(Job));
  P.off_dss = o2; o2 = align256(o2 + (size_t)(B + 1) * sizeof(int64_t));
  if (!P.segs.empty()) {
    P.off_segs = o2; o2 = align256(o2 + P.segs.size() * sizeof(Seg));
    P.off_chunks = o2; o2 = align256(o2 + P.chunks.size() * sizeof(Chunk));
    P.off_bseg = o2; o2 = align256(o2 + P.bucket_seg.size() * sizeof(int32_t));
  }
  P.off_upload_end = o2;
  P.off_var = o2; o2 = align256(o2 + (size_t)P.S * sizeof(double));
  P.off_info = o2; o2 = align256(o2 + (size_t)P.S * sizeof(double));
  P.off_status = o2; o2 = align256(o2 + (size_t)P.S * sizeof(int32_t));
  P.off_iters = o2; o2 = align256(o2 + (size_t)P.S * sizeof(int32_t));
  P.off_gws = o2; o2 = align256(o2 + P.gws_bytes);
  if (!P.segs.empty()) {
    const size_t N = (size_t)P.n_stream, NB = P.bucket_seg.size(), NC = P.chunks.size(), NS = P.segs.size();
    P.off_spl_key = o2; o2 = align256(o2 + NB * ks);
    P.off_spl_idx = o2; o2 = align256(o2 + NB * 4);
    P.off_bcnt = o2; o2 = align256(o2 + NB * 4);
    P.off_bstart = o2; o2 = align256(o2 + NB * 4);
    P.off_mat = o2; o2 = align256(o2 + (size_t)P.n_mat * 4);
    P.off_bof = o2; o2 = align256(o2 + N * 2);
    P.off_bkey = o2; o2 = align256(o2 + N * ks);
    P.off_bidx = o2; o2 = align256(o2 + N * 4);
    P.off_ranku = o2; o2 = align256(o2 + N * 4);
    P.off_rankv = o2; o2 = align256(o2 + N * 4);
    P.off_pi = o2; o2 = align256(o2 + N * 4);
    P.off_tab = o2; o2 = align256(o2 + N * rs);
    P.off_tabv = o2; o2 = align256(o2 + N * rs);
    P.off_wu = o2; o2 = align256(o2 + N * rs);
    P.off_wv = o2; o2 = align256(o2 + N * rs);
    P.off_part = o2; o2 = align256(o2 + NC * kPartStride * sizeof(double));
    P.off_state = o2; o2 = align256(o2 + NS * sizeof(SegState));
    P.off_sync = o2; o2 = align256(o2 + (5 + (size_t)kFixedPhases + 2 * ((size_t)o.max_iter + 1)) * sizeof(int32_t));
    if (ctx) {
      cudaError_t e = stream_setup(ctx->sms);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "streaming kernels setup");
    }
  }
  P.off_end = o2;
  return COPULA_SUCCESS;
}

// Whether the three families share one block table (then a plan does not
// depend on the families).
bool same_tables(const copula_ctx* ctx) {
  return !ctx || (ctx->blocks[0] == ctx->blocks[1] && ctx->blocks[1] == ctx->blocks[2]);
}

// The plan of these arguments: the context's cached plan if they are those it
// was built from, else a new one (which replaces the cached one).  Without a
// context the plan is built into `local`.
int get_plan(copula_ctx* ctx, int32_t dtype, const copula_opts& o, int32_t B, const int32_t* family,
             const int64_t* doff, const int64_t* soff, const int64_t* dss, const Plan** out, Plan& local) {
  if (!ctx || B < 1 || !doff || !soff || !dss) {
    const int rc = make_plan(ctx, dtype, o, B, family, doff, soff, dss, local);
    *out = &local;
    return rc;
  }
  if (!ctx->plan_cache) ctx->plan_cache = new PlanCache();
  PlanCache& C = *static_cast<PlanCache*>(ctx->plan_cache);
  bool hit = C.valid && C.dtype == dtype && C.B == B && std::memcmp(&C.o, &o, sizeof(o)) == 0 &&
             C.blocks_version == ctx->blocks_version && (family != nullptr) == !C.fam.empty() &&
             std::memcmp(C.doff.data(), doff, (size_t)(B + 1) * sizeof(int64_t)) == 0 &&
             std::memcmp(C.dss.data(), dss, (size_t)(B + 1) * sizeof(int64_t)) == 0;
  if (hit && family) hit = std::memcmp(C.fam.data(), family, (size_t)B * sizeof(int32_t)) == 0;
  if (hit) hit = std::memcmp(C.soff.data(), soff, C.soff.size() * sizeof(int64_t)) == 0;
  if (hit) {
    *out = &C.P;
    return COPULA_SUCCESS;
  }
  C.valid = false;
  const int rc = make_plan(ctx, dtype, o, B, family, doff, soff, dss, C.P);
  if (rc) return rc;
  C.P.id = ++ctx->next_plan_id;
  C.dtype = dtype;
  C.B = B;
  C.o = o;
  C.blocks_version = ctx->blocks_version;
  C.fam.assign(family ? family : nullptr, family ? family + B : nullptr);
  C.doff.assign(doff, doff + B + 1);
  C.dss.assign(dss, dss + B + 1);
  C.soff.assign(soff, soff + dss[B] + 1);
  C.valid = true;
  *out = &C.P;
  return COPULA_SUCCESS;
}

void free_plan_cache(copula_ctx* ctx) {
  delete static_cast<PlanCache*>(ctx->plan_cache);
  ctx->plan_cache = nullptr;
}

// The device arguments of the streaming path for an uploaded plan.
StreamArgs stream_args(const copula_ctx* ctx, const Plan& P, const copula_opts& o, int mode, const void* u,
                       const void* v, char* w) {
  StreamArgs a;
  std::memset(&a, 0, sizeof(a));
  a.u = u;
  a.v = v;
  a.segs = (const Seg*)(w + P.off_segs);
  a.nseg = (int32_t)P.segs.size();
  a.nchunk = (int32_t)P.chunks.size();
  a.chunks = (const Chunk*)(w + P.off_chunks);
  a.bucket_seg = (const int32_t*)(w + P.off_bseg);
  a.nbucket = (int32_t)P.bucket_seg.size();
  a.mode = mode;
  a.spl_key = w + P.off_spl_key;
  a.spl_idx = (uint32_t*)(w + P.off_spl_idx);
  a.bucket_cnt = (uint32_t*)(w + P.off_bcnt);
  a.bucket_start = (uint32_t*)(w + P.off_bstart);
  a.mat = (uint32_t*)(w + P.off_mat);
  a.bucket_of = (uint16_t*)(w + P.off_bof);
  a.bkey = w + P.off_bkey;
  a.bidx = (uint32_t*)(w + P.off_bidx);
  a.rank_u = (uint32_t*)(w + P.off_ranku);
  a.rank_v = (uint32_t*)(w + P.off_rankv);
  a.pi = (uint32_t*)(w + P.off_pi);
  a.tab = w + P.off_tab;
  a.tabv = w + P.off_tabv;
  a.wu = w + P.off_wu;
  a.wv = w + P.off_wv;
  a.part = (double*)(w + P.off_part);
  a.state = (SegState*)(w + P.off_state);
  a.barrier = (unsigned*)(w + P.off_sync);
  a.error = (int*)(w + P.off_sync) + 2;
  a.counter = (int32_t*)(w + P.off_sync) + 3;
  a.phase_ctr = (int32_t*)(w + P.off_sync) + 4;
  a.big_count = (int32_t*)(w + P.off_sync) + 4 + kFixedPhases + 2 * (o.max_iter + 1);
  a.nphase = kFixedPhases + 2 * (o.max_iter + 1);  // FP64: the FP32 start search's passes too
  a.barrier_spins = ctx->wait_spins > 0 ? ctx->wait_spins : (int64_t)1 << 24;
  a.barrier_phantom = ctx->wait_phantom;
  a.max_iter = o.max_iter;
  a.rtol = o.rtol;
  a.start = ctx->start;
  return a;
}

int ensure_staging(copula_ctx* ctx, size_t bytes) {
  if (ctx->staging_pending) {
    cudaError_t e = cudaEventSynchronize(ctx->staging_done);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "staging wait");
    ctx->staging_pending = false;
  }
  if (bytes <= ctx->staging_bytes) return COPULA_SUCCESS;
  if (ctx->staging) cudaFreeHost(ctx->staging);
  ctx->staging = nullptr;
  ctx->staging_bytes = 0;
  ctx->staging_plan_id = 0;
  size_t want = std::max(bytes, (size_t)1 << 16);
  cudaError_t e = cudaHostAlloc(&ctx->staging, want, cudaHostAllocDefault);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaHostAlloc staging");
  ctx->staging_bytes = want;
  return COPULA_SUCCESS;
}

int ctas_per_sm(const copula_ctx* ctx, int block, size_t smem) {
  // one CTA per SM per ~227 KB of shared memory, at most 2048 threads per SM
  size_t lim = (ctx && ctx->smem_optin) ? ctx->smem_optin : kMaxSmem;
  int by_smem = (int)std::max<size_t>(1, (lim + 1024) / (smem + 1024));
  int by_thr = std::max(1, 2048 / block);
  return std::min(by_smem, by_thr);
}

int occupancy_grid(copula_ctx* ctx, int count, int block, size_t smem) {
  return std::max(1, std::min(count, ctas_per_sm(ctx, block, smem) * ctx->sms));
}

// The host arrays of a plan's schedule and where they go in the workspace.
struct Piece {
  const void* src;
  size_t bytes, dst;
};
std::vector<Piece> schedule_pieces(const Plan& P) {
  std::vector<Piece> v = {{P.jobs.data(), P.jobs.size() * sizeof(Job), P.off_jobs},
                          {P.dss.data(), P.dss.size() * sizeof(int64_t), P.off_dss}};
  if (!P.segs.empty()) {
    v.push_back({P.segs.data(), P.segs.size() * sizeof(Seg), P.off_segs});
    v.push_back({P.chunks.data(), P.chunks.size() * sizeof(Chunk), P.off_chunks});
    v.push_back({P.bucket_seg.data(), P.bucket_seg.size() * sizeof(int32_t), P.off_bseg});
  }
  return v;
}

size_t schedule_bytes(const Plan& P) { return P.off_upload_end; }

// Copies the workspace prefix [0, off_upload_end) -- zeroed job and dataset
// counters, jobs, dataset bounds, streaming descriptors -- as one image
// through pinned memory `staging` on stream st.
void fill_schedule(const Plan& P, void* staging) {
  std::memset(staging, 0, P.off_upload_end);
  for (const Piece& q : schedule_pieces(P))
    if (q.bytes) std::memcpy((char*)staging + q.dst, q.src, q.bytes);
}

int upload_schedule(copula_ctx* ctx, const Plan& P, void* staging, char* w, cudaStream_t st) {
  fill_schedule(P, staging);
  cudaError_t e = cudaMemcpyAsync(w, staging, P.off_upload_end, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "upload schedule");
  return COPULA_SUCCESS;
}

// Uploads P's schedule image through the context's pinned staging: the image
// is built there unless the staging holds it already (a cached plan's image
// stays until another plan's replaces it, so repeat calls only copy it).
int stage_and_upload(copula_ctx* ctx, const Plan& P, char* w, cudaStream_t st) {
  if (!(P.id != 0 && ctx->staging_plan_id == P.id && ctx->staging_bytes >= schedule_bytes(P))) {
    const int rc = ensure_staging(ctx, schedule_bytes(P));  // waits for copies still reading the staging
    if (rc) return rc;
    fill_schedule(P, ctx->staging);
    ctx->staging_plan_id = P.id;
  }
  cudaError_t e = cudaMemcpyAsync(w, ctx->staging, P.off_upload_end, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->staging_done, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "upload schedule");
  ctx->staging_pending = true;
  return COPULA_SUCCESS;
}

// Enqueues the launches of an uploaded plan: counter reset, the per-bucket
// fit kernels and the combine.  Only stream operations on device memory, so
// it can be captured into a CUDA graph.
int launch_plan(copula_ctx* ctx, const Plan& P, int32_t dtype, const copula_opts& o, int mode, const void* u,
                const void* v, double* theta, double* var, int32_t* status, double* comb, const double* theta_in,
                double* l_out, double* g_out, double* h_out, char* w, cudaStream_t st, double* info,
                int32_t* iters, uint64_t* phase_ns, bool zeroed) {
  cudaError_t e = cudaSuccess;
  if (!zeroed) {  // the counters (a fresh upload brings them zeroed)
    e = cudaMemsetAsync(w + P.off_counters, 0, (kJobCounters + (size_t)P.B) * sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "memset counters");
  }

  ResidentArgs a;
  std::memset(&a, 0, sizeof(a));
  a.u = u;
  a.v = v;
  a.mode = mode;
  a.theta = theta;
  a.var = var ? var : (double*)(w + P.off_var);
  a.status = status ? status : (int32_t*)(w + P.off_status);
  a.info = info ? info : (double*)(w + P.off_info);
  a.iters = iters ? iters : (int32_t*)(w + P.off_iters);
  a.phase_ns = (unsigned long long*)phase_ns;
  a.theta_in = theta_in;
  a.l_out = l_out;
  a.g_out = g_out;
  a.h_out = h_out;
  a.max_iter = o.max_iter;
  a.rtol = o.rtol;
  a.start = ctx->start;
  // Eq. 15 by the block finishing each dataset's last subset
  a.comb = (mode == MODE_FIT) ? comb : nullptr;
  a.dss = (const int64_t*)(w + P.off_dss);
  a.ds_done = (int32_t*)(w + P.off_counters) + kJobCounters;
  a.weight = o.weight;
  const int ks = dtype == COPULA_DTYPE_F32 ? 4 : 8;
  if (ctx->timing) {
    e = cudaEventRecord(ctx->t0, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event record");
  }
  int ci = 0;
  for (const Plan::Bucket& bk : P.buckets) {
    a.jobs = (const Job*)(w + P.off_jobs) + bk.first;
    a.njobs = bk.count;
    a.counter = (int32_t*)(w + P.off_counters) + ci++;
    a.tab_in_smem = bk.tab_smem;
    a.gws = bk.gws_stride ? w + P.off_gws : nullptr;
    a.gws_stride = (int64_t)bk.gws_stride;
    a.gws_gs_off = (int64_t)bk.gws_gs_off;
    e = launch_resident(o.precision, ks, bk.block, bk.grid, bk.smem, a, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "resident launch");
    ++ctx->launches;
  }
  if (!P.segs.empty()) {
    StreamArgs sa = stream_args(ctx, P, o, mode, u, v, w);
    sa.theta = theta;
    sa.var = a.var;
    sa.status = a.status;
    sa.info = a.info;
    sa.iters = a.iters;
    sa.theta_in = theta_in;
    sa.l_out = l_out;
    sa.g_out = g_out;
    sa.h_out = h_out;
    sa.comb = a.comb;
    sa.dss = a.dss;
    sa.ds_done = a.ds_done;
    sa.weight = a.weight;
    if (ctx->timing) {
      if (!ctx->stamps) {
        e = cudaMalloc(&ctx->stamps, kStreamStamps * sizeof(unsigned long long));
        if (e != cudaSuccess) {
          ctx->stamps = nullptr;
          return cuda_fail(ctx, e, "cudaMalloc stamps");
        }
      }
      e = cudaMemsetAsync(ctx->stamps, 0, kStreamStamps * sizeof(unsigned long long), st);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "stamps reset");
      sa.stamps = ctx->stamps;
      sa.nstamps = kStreamStamps;
    }
    e = launch_stream(o.precision, ks, sa, st, ctx->timing ? ctx->sev : nullptr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "streaming launch");
    ctx->stream_timed = ctx->timing;
    ctx->launches += kStreamLaunches;
  }
  if (ctx->timing) {
    e = cudaEventRecord(ctx->t1, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event record");
    ctx->timed = true;
  }
  return COPULA_SUCCESS;
}

int run_plan(copula_ctx* ctx, const Plan& P, int32_t dtype, const copula_opts& o, int mode, const void* u,
             const void* v, double* theta, double* var, int32_t* status, double* comb, const double* theta_in,
             double* l_out, double* g_out, double* h_out, void* ws, size_t ws_bytes, cudaStream_t st,
             double* info = nullptr, int32_t* iters = nullptr, uint64_t* phase_ns = nullptr) {
  ctx->launches = 0;
  ctx->timed = false;
  ctx->stream_timed = false;
  if (!ws || ws_bytes < P.off_end) return fail(ctx, COPULA_ERR_WORKSPACE, "workspace too small");
  if (((uintptr_t)ws & 255u) != 0) return fail(ctx, COPULA_ERR_WORKSPACE, "workspace not 256-byte aligned");
  char* w = (char*)ws;
  int rc = stage_and_upload(ctx, P, w, st);
  if (rc) return rc;
  return launch_plan(ctx, P, dtype, o, mode, u, v, theta, var, status, comb, theta_in, l_out, g_out, h_out, w, st,
                     info, iters, phase_ns, true);
}

int single_plan(copula_ctx* ctx, int32_t family, int32_t dtype, const copula_opts& o, int64_t n,
                const int64_t* soff, int64_t K, const Plan** out, Plan& local) {
  if (!soff || K < 1 || n < 2) return fail(ctx, COPULA_ERR_ARG, "bad partition");
  for (int64_t k = 0; k < K; ++k)
    if (soff[k + 1] <= soff[k]) return fail(ctx, COPULA_ERR_ARG, "subset offsets not increasing");
  if (soff[K] != n) return fail(ctx, COPULA_ERR_ARG, "subset offsets must end at n");
  int64_t doff[2] = {0, n};
  int64_t dss[2] = {0, K};
  return get_plan(ctx, dtype, o, 1, &family, doff, soff, dss, out, local);
}

}  // namespace

int cop::ctx_reserve_staging(copula_ctx* ctx, size_t bytes) {
  if (!ctx) return COPULA_ERR_ARG;
  return ensure_staging(ctx, bytes);
}

extern "C" {

void copula_opts_default(copula_opts* o) {
  if (!o) return;
  o->precision = COPULA_PREC_F32C;
  o->weight = COPULA_W_INVVAR;
  o->max_iter = 64;
  o->block = 0;
  o->rtol = 0.0;  // the precision's own default (resolve_opts)
}

int copula_version(void) { return 100; }

const char* copula_last_error(copula_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

int copula_ctx_create(copula_ctx** out) {
  if (!out) return COPULA_ERR_ARG;
  copula_ctx* ctx = new copula_ctx();
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
  int optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->staging_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->t0);
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->t1);
  for (int i = 0; i < kStreamEvents && e == cudaSuccess; ++i) e = cudaEventCreate(&ctx->sev[i]);
  if (e != cudaSuccess) {
    delete ctx;
    *out = nullptr;
    return COPULA_ERR_CUDA;
  }
  ctx->smem_optin = (size_t)optin;
  build_start_tables(ctx->start);
  *out = ctx;
  return COPULA_SUCCESS;
}

int copula_ctx_destroy(copula_ctx* ctx) {
  if (!ctx) return COPULA_ERR_ARG;
  if (ctx->staging_pending) cudaEventSynchronize(ctx->staging_done);
  if (ctx->staging) cudaFreeHost(ctx->staging);
  if (ctx->rstage) cudaFreeHost(ctx->rstage);
  if (ctx->staging_done) cudaEventDestroy(ctx->staging_done);
  if (ctx->t0) cudaEventDestroy(ctx->t0);
  if (ctx->t1) cudaEventDestroy(ctx->t1);
  for (int i = 0; i < kStreamEvents; ++i)
    if (ctx->sev[i]) cudaEventDestroy(ctx->sev[i]);
  if (ctx->stamps) cudaFree(ctx->stamps);
  free_plan_cache(ctx);
  delete ctx;
  return COPULA_SUCCESS;
}

int copula_fit_workspace_size(copula_ctx* ctx, int32_t dtype, const copula_opts* opts, const int64_t* soff, int64_t K,
                              size_t* bytes) {
  if (!bytes || !soff || K < 1) return fail(ctx, COPULA_ERR_ARG, "bad arguments");
  const copula_opts o = resolve_opts(opts);
  Plan local;
  const Plan* pp = nullptr;
  int rc = single_plan(ctx, COPULA_FRANK, dtype, o, soff[K], soff, K, &pp, local);
  if (rc) return rc;
  *bytes = pp->off_end;
  if (!same_tables(ctx)) {
    // per-family block tables: the need of the most demanding family
    int64_t doff[2] = {0, soff[K]}, dss[2] = {0, K};
    for (int32_t f : {COPULA_GAUSSIAN, COPULA_GUMBEL}) {
      Plan Pf;
      rc = make_plan(ctx, dtype, o, 1, &f, doff, soff, dss, Pf);
      if (rc) return rc;
      *bytes = std::max(*bytes, Pf.off_end);
    }
  }
  return COPULA_SUCCESS;
}

int copula_fit(copula_ctx* ctx, int32_t family, int32_t dtype, const void* u, const void* v, int64_t n,
               const int64_t* soff, int64_t K, double* theta_out, double* var_out, int32_t* status_out,
               double* theta_combined_out, const copula_opts* opts, void* workspace, size_t workspace_bytes,
               void* stream) {
  if (!ctx) return COPULA_ERR_ARG;
  if (!u || !v || !theta_out) return fail(ctx, COPULA_ERR_ARG, "null pointer");
  if (family < 0 || family > 2) return fail(ctx, COPULA_ERR_ARG, "bad family");
  const copula_opts o = resolve_opts(opts);
  Plan local;
  const Plan* pp = nullptr;
  int rc = single_plan(ctx, family, dtype, o, n, soff, K, &pp, local);
  if (rc) return rc;
  const Plan& P = *pp;
  return run_plan(ctx, P, dtype, o, MODE_FIT, u, v, theta_out, var_out, status_out, theta_combined_out, nullptr,
                  nullptr, nullptr, nullptr, workspace, workspace_bytes, (cudaStream_t)stream);
}

int copula_fit_ex(copula_ctx* ctx, int32_t family, int32_t dtype, const void* u, const void* v, int64_t n,
                  const int64_t* soff, int64_t K, double* theta_out, double* var_out, int32_t* status_out,
                  double* theta_combined_out, double* info_out, int32_t* iters_out, uint64_t* phase_ns_out,
                  const copula_opts* opts, void* workspace, size_t workspace_bytes, void* stream) {
  if (!ctx) return COPULA_ERR_ARG;
  if (!u || !v || !theta_out) return fail(ctx, COPULA_ERR_ARG, "null pointer");
  if (family < 0 || family > 2) return fail(ctx, COPULA_ERR_ARG, "bad family");
  const copula_opts o = resolve_opts(opts);
  Plan local;
  const Plan* pp = nullptr;
  int rc = single_plan(ctx, family, dtype, o, n, soff, K, &pp, local);
  if (rc) return rc;
  const Plan& P = *pp;
  return run_plan(ctx, P, dtype, o, MODE_FIT, u, v, theta_out, var_out, status_out, theta_combined_out, nullptr,
                  nullptr, nullptr, nullptr, workspace, workspace_bytes, (cudaStream_t)stream, info_out, iters_out,
                  phase_ns_out);
}

int copula_ctx_set_timing(copula_ctx* ctx, int32_t on) {
  if (!ctx) return COPULA_ERR_ARG;
  ctx->timing = on != 0;
  return COPULA_SUCCESS;
}

int copula_ctx_kernel_ms(copula_ctx* ctx, double* ms) {
  if (!ctx || !ms) return COPULA_ERR_ARG;
  if (!ctx->timed) return fail(ctx, COPULA_ERR_ARG, "no timed call");
  cudaError_t e = cudaEventSynchronize(ctx->t1);
  float f = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&f, ctx->t0, ctx->t1);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "event time");
  *ms = (double)f;
  return COPULA_SUCCESS;
}

int copula_ctx_stage_ms(copula_ctx* ctx, double* ms) {
  if (!ctx || !ms) return COPULA_ERR_ARG;
  if (!ctx->stream_timed) return fail(ctx, COPULA_ERR_ARG, "the last timed call had no streaming subsets");
  cudaError_t e = cudaEventSynchronize(ctx->sev[kStreamEvents - 1]);
  for (int i = 0; i + 1 < kStreamEvents && e == cudaSuccess; ++i) {
    float f = 0.0f;
    e = cudaEventElapsedTime(&f, ctx->sev[i], ctx->sev[i + 1]);
    ms[i] = (double)f;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "event time");
  return COPULA_SUCCESS;
}

int copula_ctx_stream_stamps(copula_ctx* ctx, uint64_t* ns_out, int32_t cap, int32_t* count) {
  if (!ctx || !ns_out || !count || cap < 0) return COPULA_ERR_ARG;
  if (!ctx->stream_timed || !ctx->stamps) return fail(ctx, COPULA_ERR_ARG, "the last timed call had no streaming subsets");
  cudaError_t e = cudaEventSynchronize(ctx->sev[kStreamEvents - 1]);
  unsigned long long h[kStreamStamps];
  if (e == cudaSuccess) e = cudaMemcpy(h, ctx->stamps, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stamps read");
  int n = 0;
  while (n < kStreamStamps && h[n] != 0ull) ++n;
  for (int i = 0; i < n && i < cap; ++i) ns_out[i] = (uint64_t)h[i];
  *count = n;
  return COPULA_SUCCESS;
}

int copula_ctx_launches(copula_ctx* ctx, int32_t* launches) {
  if (!ctx || !launches) return COPULA_ERR_ARG;
  *launches = ctx->launches;
  return COPULA_SUCCESS;
}

struct copula_plan {
  copula_ctx* ctx = nullptr;
  Plan P;
  int32_t dtype = 0;
  copula_opts o;
  void* staging = nullptr;  // pinned copy of the schedule, owned by the plan
};

int copula_plan_create(copula_ctx* ctx, copula_plan** out, int32_t B, const int32_t* family, int32_t dtype,
                       const int64_t* doff, const int64_t* soff, const int64_t* dss, const copula_opts* opts,
                       size_t* workspace_bytes) {
  if (!ctx || !out || !family) return fail(ctx, COPULA_ERR_ARG, "bad arguments");
  copula_plan* p = new copula_plan();
  p->ctx = ctx;
  p->dtype = dtype;
  p->o = resolve_opts(opts);
  int rc = make_plan(ctx, dtype, p->o, B, family, doff, soff, dss, p->P);
  if (rc) {
    delete p;
    return rc;
  }
  if (cudaHostAlloc(&p->staging, std::max<size_t>(schedule_bytes(p->P), 256), cudaHostAllocDefault) != cudaSuccess) {
    delete p;
    return fail(ctx, COPULA_ERR_CUDA, "cudaHostAlloc plan staging");
  }
  if (workspace_bytes) *workspace_bytes = p->P.off_end;
  *out = p;
  return COPULA_SUCCESS;
}

int copula_plan_upload(copula_plan* p, void* workspace, size_t workspace_bytes, void* stream) {
  if (!p) return COPULA_ERR_ARG;
  if (!workspace || workspace_bytes < p->P.off_end || ((uintptr_t)workspace & 255u) != 0)
    return fail(p->ctx, COPULA_ERR_WORKSPACE, "workspace too small or misaligned");
  return upload_schedule(p->ctx, p->P, p->staging, (char*)workspace, (cudaStream_t)stream);
}

int copula_plan_run(copula_plan* p, const void* u, const void* v, double* theta_out, double* var_out,
                    int32_t* status_out, double* theta_combined_out, void* workspace, size_t workspace_bytes,
                    void* stream) {
  if (!p) return COPULA_ERR_ARG;
  if (!u || !v || !theta_out) return fail(p->ctx, COPULA_ERR_ARG, "null pointer");
  if (!workspace || workspace_bytes < p->P.off_end || ((uintptr_t)workspace & 255u) != 0)
    return fail(p->ctx, COPULA_ERR_WORKSPACE, "workspace too small or misaligned");
  p->ctx->launches = 0;
  p->ctx->timed = false;
  p->ctx->stream_timed = false;
  return launch_plan(p->ctx, p->P, p->dtype, p->o, MODE_FIT, u, v, theta_out, var_out, status_out,
                     theta_combined_out, nullptr, nullptr, nullptr, nullptr, (char*)workspace, (cudaStream_t)stream,
                     nullptr, nullptr, nullptr, false);
}

int copula_plan_diagnostics(copula_plan* p, const void* workspace, size_t workspace_bytes, double* info_out,
                            int32_t* iters_out, void* stream) {
  if (!p) return COPULA_ERR_ARG;
  if (!workspace || workspace_bytes < p->P.off_end || ((uintptr_t)workspace & 255u) != 0)
    return fail(p->ctx, COPULA_ERR_WORKSPACE, "workspace too small or misaligned");
  const char* w = (const char*)workspace;
  const size_t S = (size_t)p->P.S;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (info_out) e = cudaMemcpyAsync(info_out, w + p->P.off_info, S * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && iters_out)
    e = cudaMemcpyAsync(iters_out, w + p->P.off_iters, S * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(p->ctx, e, "plan diagnostics copy");
  return COPULA_SUCCESS;
}

int copula_plan_destroy(copula_plan* p) {
  if (!p) return COPULA_ERR_ARG;
  if (p->staging) cudaFreeHost(p->staging);
  delete p;
  return COPULA_SUCCESS;
}

static int parse_blocks(copula_ctx* ctx, const int32_t* m_max, const int32_t* threads, int32_t count,
                        std::vector<std::pair<int32_t, int32_t>>& b) {
  if (!ctx || count < 0 || (count > 0 && (!m_max || !threads))) return COPULA_ERR_ARG;
  for (int32_t i = 0; i < count; ++i) {
    if (threads[i] != 128 && threads[i] != 256 && threads[i] != 512) return fail(ctx, COPULA_ERR_ARG, "bad block");
    if (i > 0 && m_max[i] <= m_max[i - 1]) return fail(ctx, COPULA_ERR_ARG, "bucket bounds not increasing");
    b.emplace_back(m_max[i], threads[i]);
  }
  return COPULA_SUCCESS;
}

int copula_ctx_set_blocks(copula_ctx* ctx, const int32_t* m_max, const int32_t* threads, int32_t count) {
  std::vector<std::pair<int32_t, int32_t>> b;
  const int rc = parse_blocks(ctx, m_max, threads, count, b);
  if (rc) return rc;
  for (auto& t : ctx->blocks) t = b;
  ++ctx->blocks_version;
  return COPULA_SUCCESS;
}

int copula_ctx_set_wait_limit(copula_ctx* ctx, int64_t spins, int32_t phantom_arrivals) {
  if (!ctx || spins < 0 || phantom_arrivals < 0 || phantom_arrivals > 1) return COPULA_ERR_ARG;
  ctx->wait_spins = spins;
  ctx->wait_phantom = phantom_arrivals;
  return COPULA_SUCCESS;
}

int copula_ctx_set_family_blocks(copula_ctx* ctx, int32_t family, const int32_t* m_max, const int32_t* threads,
                                 int32_t count) {
  if (family < 0 || family > 2) return fail(ctx, COPULA_ERR_ARG, "bad family");
  std::vector<std::pair<int32_t, int32_t>> b;
  const int rc = parse_blocks(ctx, m_max, threads, count, b);
  if (rc) return rc;
  ctx->blocks[family] = b;
  ++ctx->blocks_version;
  return COPULA_SUCCESS;
}

int copula_fit_batch_workspace_size(copula_ctx* ctx, int32_t dtype, const copula_opts* opts, int32_t B,
                                    const int32_t* family, const int64_t* doff, const int64_t* soff,
                                    const int64_t* dss, size_t* bytes) {
  if (!bytes) return fail(ctx, COPULA_ERR_ARG, "bad arguments");
  if (!family && !same_tables(ctx)) return fail(ctx, COPULA_ERR_ARG, "families needed with per-family block tables");
  const copula_opts o = resolve_opts(opts);
  Plan local;
  const Plan* pp = nullptr;
  int rc = get_plan(ctx, dtype, o, B, family, doff, soff, dss, &pp, local);
  if (rc) return rc;
  *bytes = pp->off_end;
  return COPULA_SUCCESS;
}

int copula_fit_batch(copula_ctx* ctx, int32_t B, const int32_t* family, int32_t dtype, const void* u, const void* v,
                     const int64_t* doff, const int64_t* soff, const int64_t* dss, double* theta_out, double* var_out,
                     int32_t* status_out, double* theta_combined_out, const copula_opts* opts, void* workspace,
                     size_t workspace_bytes, void* stream) {
  if (!ctx) return COPULA_ERR_ARG;
  if (!u || !v || !theta_out || !family) return fail(ctx, COPULA_ERR_ARG, "null pointer");
  const copula_opts o = resolve_opts(opts);
  Plan local;
  const Plan* pp = nullptr;
  int rc = get_plan(ctx, dtype, o, B, family, doff, soff, dss, &pp, local);
  if (rc) return rc;
  const Plan& P = *pp;
  return run_plan(ctx, P, dtype, o, MODE_FIT, u, v, theta_out, var_out, status_out, theta_combined_out, nullptr,
                  nullptr, nullptr, nullptr, workspace, workspace_bytes, (cudaStream_t)stream);
}

// Host-buffer layout after the fit workspace: u, v, then the results in one
// block (theta S, var S, combined B as doubles; status S int32) so that a
// single copy brings them back.
static size_t host_results_bytes(int64_t S, int64_t B) {
  return (size_t)(2 * S + B) * sizeof(double) + (size_t)S * sizeof(int32_t);
}

static size_t host_workspace_bytes(size_t fit_bytes, int32_t dtype, int64_t n, int64_t S, int64_t B) {
  const size_t es = dtype == COPULA_DTYPE_F32 ? 4 : 8;
  return align256(fit_bytes) + 2 * align256((size_t)n * es) + align256(host_results_bytes(S, B));
}

int copula_fit_host_workspace_size(copula_ctx* ctx, int32_t dtype, const copula_opts* opts, const int64_t* soff,
                                   int64_t K, size_t* bytes) {
  size_t b = 0;
  int rc = copula_fit_workspace_size(ctx, dtype, opts, soff, K, &b);
  if (rc) return rc;
  *bytes = host_workspace_bytes(b, dtype, soff[K], K, 1);
  return COPULA_SUCCESS;
}

int copula_fit_batch_host_workspace_size(copula_ctx* ctx, int32_t dtype, const copula_opts* opts, int32_t B,
                                         const int32_t* family, const int64_t* doff, const int64_t* soff,
                                         const int64_t* dss, size_t* bytes) {
  size_t b = 0;
  int rc = copula_fit_batch_workspace_size(ctx, dtype, opts, B, family, doff, soff, dss, &b);
  if (rc) return rc;
  *bytes = host_workspace_bytes(b, dtype, doff[B], dss[B], B);
  return COPULA_SUCCESS;
}

// The device address of page-locked host memory the device can read (UVA:
// the host address itself), or null for pageable memory.
static const void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

// A planned fit on host buffers: inputs to the GPU (or read in place from
// mapped pinned memory), the fit, one copy of all results back through the
// context's pinned staging, and a wait on the stream.
static int run_host(copula_ctx* ctx, const Plan& P, int32_t dtype, const copula_opts& o, const void* u_host,
                    const void* v_host, double* theta_out, double* var_out, int32_t* status_out,
                    double* theta_combined_out, void* workspace, size_t workspace_bytes, cudaStream_t st) {
  const int64_t n = P.n, S = P.S, B = P.B;
  const size_t es = dtype == COPULA_DTYPE_F32 ? 4 : 8;
  const size_t rb = host_results_bytes(S, B);
  size_t off = align256(P.off_end);
  char* w = (char*)workspace;
  char* du = w + off;
  off += align256((size_t)n * es);
  char* dv = w + off;
  off += align256((size_t)n * es);
  char* dres = w + off;
  off += align256(rb);
  if (!workspace || workspace_bytes < off) return fail(ctx, COPULA_ERR_WORKSPACE, "workspace too small");
  if (((uintptr_t)workspace & 255u) != 0) return fail(ctx, COPULA_ERR_WORKSPACE, "workspace not 256-byte aligned");
  if (ctx->rstage_bytes < rb) {
    if (ctx->rstage) cudaFreeHost(ctx->rstage);
    ctx->rstage = nullptr;
    ctx->rstage_bytes = 0;
    const size_t want = std::max(rb, (size_t)1 << 16);
    cudaError_t e = cudaHostAlloc(&ctx->rstage, want, cudaHostAllocDefault);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaHostAlloc results staging");
    ctx->rstage_bytes = want;
  }
  double* dth = (double*)dres;
  double* dvar = dth + S;
  double* dcomb = dvar + S;
  int32_t* dst = (int32_t*)(dcomb + B);
  // The shared-memory path reads each input element once, coalesced: from
  // device-addressable pinned host memory it reads them over the host link
  // itself, with no staging copy in front of the kernel.
  const void* ku = P.segs.empty() ? mapped_host(u_host) : nullptr;
  const void* kv = P.segs.empty() ? mapped_host(v_host) : nullptr;
  cudaError_t e = cudaSuccess;
  if (!ku || !kv) {
    e = cudaMemcpyAsync(du, u_host, (size_t)n * es, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dv, v_host, (size_t)n * es, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "H2D inputs");
    ku = du;
    kv = dv;
  }
  int rc = run_plan(ctx, P, dtype, o, MODE_FIT, ku, kv, dth, dvar, dst, dcomb, nullptr, nullptr, nullptr, nullptr,
                    workspace, P.off_end, st);
  if (rc) return rc;
  e = cudaMemcpyAsync(ctx->rstage, dres, rb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "D2H results");
  const double* h = (const double*)ctx->rstage;
  std::memcpy(theta_out, h, (size_t)S * sizeof(double));
  if (var_out) std::memcpy(var_out, h + S, (size_t)S * sizeof(double));
  if (theta_combined_out) std::memcpy(theta_combined_out, h + 2 * S, (size_t)B * sizeof(double));
  if (status_out) std::memcpy(status_out, (const int32_t*)(h + 2 * S + B), (size_t)S * sizeof(int32_t));
  return COPULA_SUCCESS;
}

int copula_fit_host(copula_ctx* ctx, int32_t family, int32_t dtype, const void* u_host, const void* v_host, int64_t n,
                    const int64_t* soff, int64_t K, double* theta_out, double* var_out, int32_t* status_out,
                    double* theta_combined_out, const copula_opts* opts, void* workspace, size_t workspace_bytes,
                    void* stream) {
  if (!ctx) return COPULA_ERR_ARG;
  if (!u_host || !v_host || !theta_out || !soff || K < 1) return fail(ctx, COPULA_ERR_ARG, "null pointer");
  if (family < 0 || family > 2) return fail(ctx, COPULA_ERR_ARG, "bad family");
  const copula_opts o = resolve_opts(opts);
  Plan local;
  const Plan* pp = nullptr;
  int rc = single_plan(ctx, family, dtype, o, n, soff, K, &pp, local);
  if (rc) return rc;
  const Plan& P = *pp;
  return run_host(ctx, P, dtype, o, u_host, v_host, theta_out, var_out, status_out, theta_combined_out, workspace,
                  workspace_bytes, (cudaStream_t)stream);
}

int copula_fit_batch_host(copula_ctx* ctx, int32_t B, const int32_t* family, int32_t dtype, const void* u_host,
                          const void* v_host, const int64_t* doff, const int64_t* soff, const int64_t* dss,
                          double* theta_out, double* var_out, int32_t* status_out, double* theta_combined_out,
                          const copula_opts* opts, void* workspace, size_t workspace_bytes, void* stream) {
  if (!ctx) return COPULA_ERR_ARG;
  if (!u_host || !v_host || !theta_out || !family) return fail(ctx, COPULA_ERR_ARG, "null pointer");
  const copula_opts o = resolve_opts(opts);
  Plan local;
  const Plan* pp = nullptr;
  int rc = get_plan(ctx, dtype, o, B, family, doff, soff, dss, &pp, local);
  if (rc) return rc;
  const Plan& P = *pp;
  return run_host(ctx, P, dtype, o, u_host, v_host, theta_out, var_out, status_out, theta_combined_out, workspace,
                  workspace_bytes, (cudaStream_t)stream);
}

int copula_ranks(copula_ctx* ctx, int32_t dtype, const void* x, int64_t n, const int64_t* soff, int64_t K,
                 int32_t* ranks_out, void* workspace, size_t workspace_bytes, void* stream) {
  if (!ctx) return COPULA_ERR_ARG;
  if (!x || !ranks_out) return fail(ctx, COPULA_ERR_ARG, "null pointer");
  copula_opts o;
  copula_opts_default(&o);
  Plan local;
  const Plan* pp = nullptr;
  int rc = single_plan(ctx, COPULA_FRANK, dtype, o, n, soff, K, &pp, local);
  if (rc) return rc;
  const Plan& P = *pp;
  if (!workspace || workspace_bytes < P.off_end) return fail(ctx, COPULA_ERR_WORKSPACE, "workspace too small");
  char* w = (char*)workspace;
  cudaStream_t st = (cudaStream_t)stream;
  rc = stage_and_upload(ctx, P, w, st);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  const int ks = dtype == COPULA_DTYPE_F32 ? 4 : 8;
  int ci = 0;
  for (const Plan::Bucket& bk : P.buckets) {
    const size_t smem = res_layout(bk.m_max, ks, 4, false, false, bk.block).total;
    const int grid = occupancy_grid(ctx, bk.count, bk.block, smem);
    e = launch_ranks(ks, bk.block, grid, smem, x, (const Job*)(w + P.off_jobs) + bk.first, bk.count,
                     (int32_t*)(w + P.off_counters) + ci++, ranks_out, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ranks launch");
  }
  if (!P.segs.empty()) {
    e = launch_stream_ranks(ks, stream_args(ctx, P, o, MODE_FIT, x, x, w), x, ranks_out, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "streaming ranks launch");
  }
  return COPULA_SUCCESS;
}

int copula_rank_corr(copula_ctx* ctx, int32_t dtype, const void* u, const void* v, int64_t n, const int64_t* soff,
                     int64_t K, double* tau_out, double* rho_out, void* workspace, size_t workspace_bytes,
                     void* stream) {
  if (!ctx) return COPULA_ERR_ARG;
  if (!u || !v || !tau_out || !rho_out) return fail(ctx, COPULA_ERR_ARG, "null pointer");
  copula_opts o;
  copula_opts_default(&o);
  Plan local;
  const Plan* pp = nullptr;
  int rc = single_plan(ctx, COPULA_FRANK, dtype, o, n, soff, K, &pp, local);
  if (rc) return rc;
  const Plan& P = *pp;
  if (!workspace || workspace_bytes < P.off_end) return fail(ctx, COPULA_ERR_WORKSPACE, "workspace too small");
  char* w = (char*)workspace;
  cudaStream_t st = (cudaStream_t)stream;
  rc = stage_and_upload(ctx, P, w, st);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  const int ks = dtype == COPULA_DTYPE_F32 ? 4 : 8;
  int ci = 0;
  for (const Plan::Bucket& bk : P.buckets) {
    const size_t smem = res_layout(bk.m_max, ks, 4, false, false, bk.block).total;
    const int grid = occupancy_grid(ctx, bk.count, bk.block, smem);
    e = launch_rankcorr(ks, bk.block, grid, smem, u, v, (const Job*)(w + P.off_jobs) + bk.first, bk.count,
                        (int32_t*)(w + P.off_counters) + ci++, tau_out, rho_out, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rank correlation launch");
  }
  if (!P.segs.empty()) {
    e = launch_stream_rank_corr(ks, stream_args(ctx, P, o, MODE_FIT, u, v, w), tau_out, rho_out, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "streaming rank correlation launch");
  }
  return COPULA_SUCCESS;
}

int copula_loglik(copula_ctx* ctx, int32_t family, int32_t dtype, const void* u, const void* v, int64_t n,
                  const int64_t* soff, int64_t K, const double* theta_in, double* l_out, double* g_out, double* h_out,
                  const copula_opts* opts, void* workspace, size_t workspace_bytes, void* stream) {
  if (!ctx) return COPULA_ERR_ARG;
  if (!u || !v || !theta_in) return fail(ctx, COPULA_ERR_ARG, "null pointer");
  if (family < 0 || family > 2) return fail(ctx, COPULA_ERR_ARG, "bad family");
  const copula_opts o = resolve_opts(opts);
  Plan local;
  const Plan* pp = nullptr;
  int rc = single_plan(ctx, family, dtype, o, n, soff, K, &pp, local);
  if (rc) return rc;
  const Plan& P = *pp;
  return run_plan(ctx, P, dtype, o, MODE_LOGLIK, u, v, nullptr, nullptr, nullptr, nullptr, theta_in, l_out, g_out,
                  h_out, workspace, workspace_bytes, (cudaStream_t)stream);
}

}  // extern "C"

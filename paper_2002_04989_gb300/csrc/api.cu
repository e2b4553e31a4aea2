// C ABI of libeeid: argument validation, planning of the task lists, workspace
// management inside the context's HBM budget, and the launch sequence
//   K-a tridiag (A and minors) -> K-b bisect (A) -> denominators -> K-b bisect
//   (minors, interlacing brackets) -> K-c identity.
// Every arithmetic step runs in the CUDA kernels; the host only plans and launches.
#include "eeid.h"
#include "host_plan.h"
#include "internal.cuh"

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace eeid {
int tridiag_blocks_per_sm(bool smem_path, int warps, int max_m, bool hi);
cudaError_t launch_tridiag_cluster(int warps, int nclusters, int csize, const TridiagLaunch& L,
                                   cudaStream_t s);
int tridiag_max_active_clusters(int warps, int csize, int max_m);
cudaError_t launch_tridiag_group(int warps, int ngroups, int group, const TridiagLaunch& L,
                                 cudaStream_t s);
int tridiag_group_blocks_per_sm(int warps, int max_m);
cudaError_t launch_tridiag_group_short(const TridiagLaunch& L, cudaStream_t s);
size_t tridiag_herm_slot_doubles(int max_m);
size_t tridiag_herm_smem_bytes(int max_m, int warps);
cudaError_t launch_tridiag_herm(int warps, int grid, const TridiagLaunch& L, cudaStream_t s);
cudaError_t preload_tridiag_herm();
int tridiag_herm_blocks_per_sm(int warps, int max_m);
cudaError_t preload_vectors();
size_t pick_refs_smem_bytes(int nrows, int n);
cudaError_t launch_pick_refs(const double* g, int nrows, int n, int* refs, int* row_ref,
                             int* nref, unsigned char* need, cudaStream_t s);
cudaError_t launch_signed(const void* rows, int nrows, int n, cudaStream_t s);
size_t signed_row_bytes();
void fill_signed_row(void* dst, const double* g, const double* q, const int* pos, double* out,
                     int ref);
}

using namespace eeid;

namespace {

thread_local std::string g_err;

}  // namespace

namespace eeid {
// Lets other translation units report through eeid_last_error().
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace eeid

namespace {

eeid_status fail(eeid_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

eeid_status cuda_fail(cudaError_t e, const char* what) {
  return fail(EEID_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define EEID_CK(call, what)                         \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

constexpr size_t kAlign = 256;
constexpr int kStatusSlots = 64;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

}  // namespace

struct eeid_ctx {
  int device = 0;
  int sms = 0;
  size_t budget = 0;
  char* ws = nullptr;
  size_t ws_cap = 0;
  // Device status words, one per stream the context has run on (slot 0: internal work
  // and streams beyond the table), so eeid_sync(stream) reads and clears only the word of
  // that stream's calls.  h_status: pinned copies read back on the stream itself.
  unsigned* d_status = nullptr;
  unsigned* h_status = nullptr;
  std::vector<cudaStream_t> status_streams;   // slot s + 1 belongs to status_streams[s]
  // eeid_components_host: device copies of A, the grid and the eigenvalues, kept for
  // the next call (no allocation per call once it is large enough).
  char* host_call_buf = nullptr;
  size_t host_call_cap = 0;
  char* h_stage = nullptr;
  size_t h_stage_cap = 0;
  cudaEvent_t stage_ev = nullptr;
  bool stage_used = false;
  int64_t launches = 0;
  int occ_cache[3][17] = {};  // blocks/SM per (path, warps) at the last max_m
  int occ_m[3][17] = {};
  // path: 0 = working matrix in shared memory, 1 = global slot, 2 = global slot built
  // for high occupancy
  struct Rule { int lo, hi; int path; int warps; };
  std::vector<Rule> rules;  // tuning overrides, later ones win
  int rules_version = 0;
  // CUDA graphs of batched calls, keyed by the full description of the batch.
  struct GraphEntry {
    std::string key;
    cudaGraphExec_t exec = nullptr;
    char* pinned = nullptr;  // this graph's own copy of the uploaded metadata
    int nkernels = 0;
    uint64_t last_use = 0;
  };
  std::vector<GraphEntry> graphs;
  uint64_t graph_clock = 0;
  cudaStream_t cap_stream = nullptr;
  bool graphs_enabled = true;
  // Tail overlap: the last round of a multi-round tridiagonalisation runs on aux_stream
  // (greatest priority) while the caller's stream bisects the finished matrices.
  bool overlap_enabled = true;
  // Round launches (serving): each group's persistent reduction is cut into launches
  // of at most one round of tasks, so kernels of other streams get SMs between them.
  bool round_launches = false;
  // SMs the persistent reductions leave free (serving: room for a second batch).
  int sm_reserve = 0;
  // Cluster plan for groups of few large reductions (see cluster_size_for), and the group
  // plan for the fewest largest (see group_size_for).
  bool clusters_enabled = true;
  bool groups_enabled = true;
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  bool timing = false;
  cudaEvent_t ev[EEID_NUM_PHASES][2] = {};
  bool ran[EEID_NUM_PHASES] = {};
  // eeid_eigenvectors: its device buffers (magnitudes, rotated components, references)
  // and a pinned buffer for the references read back and the rows uploaded.
  char* vbuf = nullptr;
  size_t vbuf_cap = 0;
  char* h_vec = nullptr;
  size_t h_vec_cap = 0;
  cudaEvent_t vec_ev = nullptr;
  bool vec_used = false;
  int64_t vec_refs = 0;
};

namespace {

// ------------------------------------------------------------------ planning

// Tridiagonalisation configuration by matrix size (shared memory resident up to
// kTridiagSmemMaxM, global slots above).  Depends on m only, so a matrix's result
// never depends on what else is in the batch.
struct TriCfg {
  bool smem;
  int warps;
  bool herm = false;   // complex Hermitian reduction (its own kernel, global slots)
  bool hi = false;     // high-occupancy build of the global-slot variant
};
inline TriCfg cfg_of(int path, int warps) { return {path == 0, warps, false, path == 2}; }
inline int path_of(const TriCfg& c) { return c.smem ? 0 : c.hi ? 2 : 1; }
constexpr int kHermMaxM = 2048;   // largest complex Hermitian matrix (shared-memory vectors)
constexpr size_t kMaxSmemPerBlock = 232448;  // opt-in shared memory per CTA on sm_103a

TriCfg tri_cfg_default(int m) {
  if (m <= 32) return {true, 1};
  if (m <= 64) return {true, 2};
  if (m <= kTridiagSmemMaxM) return {true, 4};
  if (m <= 512) return {false, 4};
  if (tridiag_smem_bytes(false, m, 16) <= kMaxSmemPerBlock) return {false, 16};
  if (tridiag_smem_bytes(false, m, 12) <= kMaxSmemPerBlock) return {false, 12};
  return {false, 8};
}
inline int cfg_key(const TriCfg& c) {
  return c.herm ? 96 + c.warps : c.hi ? 64 + c.warps : (c.smem ? 0 : 32) + c.warps;
}

// Warps per CTA of the cluster variant for m x m matrices: the most that fit.
int cluster_warps(int m) {
  for (int w : {16, 12, 8})
    if (tridiag_smem_bytes(false, m, w) <= kMaxSmemPerBlock) return w;
  return 0;
}

TriCfg herm_cfg(int m) {
  return {false, tridiag_herm_smem_bytes(m, 8) <= kMaxSmemPerBlock ? 8 : 4, true};
}

bool cfg_supported(int path, int warps, int m) {
  bool ok;
  if (path == 0) ok = (warps == 1 || warps == 2 || warps == 4 || warps == 8) && m <= kTridiagSmemMaxM;
  else if (path == 1)
    ok = (warps == 1 || warps == 2 || warps == 4 || warps == 8 || warps == 12 || warps == 16) &&
         m <= kTridiagMaxM;
  else if (path == 2) ok = (warps == 4 || warps == 8) && m <= kTridiagMaxM;
  else ok = false;
  return ok && tridiag_smem_bytes(path == 0, m, warps) <= kMaxSmemPerBlock;
}

struct Problem {
  const double* dA;
  int64_t lda;
  int n;
  std::vector<int> rows;  // eigen-indices
  std::vector<int> cols;  // component indices
  double* out;            // nrows x ncols (may be null for eig-only modes)
  double* lam_user;       // optional
  double* mu_user;        // minor-eigvals mode output (ncols x (n-1))
  bool all_rows = false;  // rows / cols given as NULL ("all")
  bool all_cols = false;
  // Sign recovery: every minor of this problem is the rotated minor of (rot, j)
  // (see TridiagTask); rot is never among the cols.
  int rot = -1;
  // Eigenvalues of A computed earlier on the same stream: A is not reduced or bisected
  // again, and these seed the minors' brackets and the denominators.
  const double* lam_in = nullptr;
  // Complex Hermitian A (interleaved re/im doubles, lda in complex elements).
  bool herm = false;
};

enum Mode { MODE_EIGVALS, MODE_MINORS, MODE_COMPONENTS };

struct Arena {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return o;
  }
};

eeid_status check_ctx(eeid_ctx* ctx) {
  if (!ctx) return fail(EEID_ERR_INVALID, "null context");
  return EEID_OK;
}

eeid_status parse_indices(const int64_t* h, int64_t cnt, int64_t n, const char* what,
                          std::vector<int>& out) {
  if (cnt < 0) return fail(EEID_ERR_INVALID, "%s: negative count", what);
  if (!h) {
    if (cnt != n) return fail(EEID_ERR_INVALID, "%s: NULL means all, count must equal n", what);
    out.resize(n);
    for (int64_t k = 0; k < n; ++k) out[k] = (int)k;
    return EEID_OK;
  }
  out.resize(cnt);
  std::vector<char> seen(n > 0 ? n : 1, 0);
  for (int64_t k = 0; k < cnt; ++k) {
    const int64_t v = h[k];
    if (v < 0 || v >= n) return fail(EEID_ERR_INVALID, "%s[%lld] = %lld out of [0, %lld)", what,
                                     (long long)k, (long long)v, (long long)n);
    if (seen[v]) return fail(EEID_ERR_INVALID, "%s: duplicate index %lld", what, (long long)v);
    seen[v] = 1;
    out[k] = (int)v;
  }
  return EEID_OK;
}

eeid_status check_matrix(const double* dA, int64_t lda, int64_t n) {
  if (n < 0) return fail(EEID_ERR_INVALID, "n = %lld < 0", (long long)n);
  if (n > kTridiagMaxM) return fail(EEID_ERR_INVALID, "n = %lld exceeds the limit %d",
                                    (long long)n, kTridiagMaxM);
  if (n > 0 && !dA) return fail(EEID_ERR_INVALID, "matrix pointer is NULL");
  if (n > 0 && lda < n) return fail(EEID_ERR_INVALID, "lda = %lld < n = %lld", (long long)lda,
                                    (long long)n);
  return EEID_OK;
}

void clear_graphs(eeid_ctx* ctx) {
  for (auto& g : ctx->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.pinned) cudaFreeHost(g.pinned);
  }
  ctx->graphs.clear();
}

eeid_status ensure_ws(eeid_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_cap) return EEID_OK;
  if (bytes > ctx->budget)
    return fail(EEID_ERR_NOMEM, "workspace of %zu bytes exceeds the HBM budget of %zu bytes", bytes,
                ctx->budget);
  clear_graphs(ctx);  // graphs bake in workspace addresses
  if (ctx->ws) {
    cudaError_t e = cudaFree(ctx->ws);  // synchronises the device: prior work is done
    ctx->ws = nullptr;
    ctx->ws_cap = 0;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree(workspace)");
  }
  size_t cap = std::min(ctx->budget, std::max(bytes, (size_t)64 << 20));
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(EEID_ERR_NOMEM, "cudaMalloc(%zu) failed: %s", cap, cudaGetErrorString(e));
  }
  ctx->ws = (char*)p;
  ctx->ws_cap = cap;
  return EEID_OK;
}

eeid_status ensure_stage(eeid_ctx* ctx, size_t bytes) {
  if (ctx->stage_used) {
    // the previous call's metadata copy must have left the staging buffer
    cudaError_t e = cudaEventSynchronize(ctx->stage_ev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize(stage)");
  }
  if (bytes <= ctx->h_stage_cap) return EEID_OK;
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  ctx->h_stage = nullptr;
  size_t cap = std::max(bytes, (size_t)1 << 20);
  cudaError_t e = cudaMallocHost((void**)&ctx->h_stage, cap);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost(stage)");
  ctx->h_stage_cap = cap;
  return EEID_OK;
}

// The context's greatest-priority stream and its fork/join events (tail overlap).
eeid_status ensure_aux(eeid_ctx* ctx) {
  if (ctx->aux_stream) return EEID_OK;
  int least = 0, greatest = 0;
  EEID_CK(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priority range");
  EEID_CK(cudaStreamCreateWithPriority(&ctx->aux_stream, cudaStreamNonBlocking, greatest),
          "aux stream");
  EEID_CK(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming), "fork event");
  EEID_CK(cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming), "join event");
  return EEID_OK;
}

// Status slot of a stream (assigned at its first use; slot 0 when the table is full).
int status_slot(eeid_ctx* ctx, cudaStream_t s, bool assign) {
  for (size_t k = 0; k < ctx->status_streams.size(); ++k)
    if (ctx->status_streams[k] == s) return (int)k + 1;
  if (!assign || (int)ctx->status_streams.size() + 1 >= kStatusSlots) return 0;
  ctx->status_streams.push_back(s);
  return (int)ctx->status_streams.size();
}

TriCfg tri_cfg(const eeid_ctx* ctx, int m) {
  for (auto it = ctx->rules.rbegin(); it != ctx->rules.rend(); ++it)
    if (m >= it->lo && m <= it->hi && cfg_supported(it->path, it->warps, m))
      return cfg_of(it->path, it->warps);
  return tri_cfg_default(m);
}

bool rule_covers(const eeid_ctx* ctx, int m) {
  for (const auto& r : ctx->rules)
    if (m >= r.lo && m <= r.hi) return true;
  return false;
}



int blocks_per_sm(eeid_ctx* ctx, const TriCfg& c, int max_m) {
  if (c.herm) return std::max(1, tridiag_herm_blocks_per_sm(c.warps, max_m));
  int& cache = ctx->occ_cache[path_of(c)][c.warps];
  int& cm = ctx->occ_m[path_of(c)][c.warps];
  if (cache == 0 || cm != max_m) {
    cache = std::max(1, tridiag_blocks_per_sm(c.smem, c.warps, max_m, c.hi));
    cm = max_m;
  }
  return cache;
}

// Everything that determines a batched call's task lists and device pointers; two
// calls with equal keys can replay the same CUDA graph.
std::string batch_key(const std::vector<Problem>& probs, bool timing, int rules_version,
                      int plan_flags) {
  std::string k;
  auto put = [&](const void* p, size_t n) { k.append((const char*)p, n); };
  const int hdr[4] = {timing ? 1 : 0, rules_version, (int)probs.size(), plan_flags};
  put(hdr, sizeof hdr);
  for (const Problem& P : probs) {
    put(&P.dA, sizeof P.dA);
    put(&P.lda, sizeof P.lda);
    put(&P.n, sizeof P.n);
    put(&P.out, sizeof P.out);
    put(&P.lam_user, sizeof P.lam_user);
    put(&P.rot, sizeof P.rot);
    put(&P.herm, sizeof P.herm);
    put(&P.lam_in, sizeof P.lam_in);
    const int nr = (int)P.rows.size(), nc = (int)P.cols.size();
    const char flags = (char)((P.all_rows ? 1 : 0) | (P.all_cols ? 2 : 0));
    put(&flags, 1);
    put(&nr, sizeof nr);
    put(&nc, sizeof nc);
    if (!P.all_rows) put(P.rows.data(), sizeof(int) * nr);
    if (!P.all_cols) put(P.cols.data(), sizeof(int) * nc);
  }
  return k;
}

constexpr size_t kMaxGraphs = 8;

// Plan, upload and launch the whole path for a list of problems.  With `ge` set, the
// metadata goes to that graph entry's own pinned buffer and the upload and every
// launch are captured (on the context's capture stream) into ge->exec instead of
// being enqueued on `stream`; the caller then launches the graph.
eeid_status run(eeid_ctx* ctx, std::vector<Problem>& probs, Mode mode, cudaStream_t stream,
                eeid_ctx::GraphEntry* ge = nullptr) {
  EEID_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  unsigned* const status_word = ctx->d_status + status_slot(ctx, stream, true);
  // ---- task lists (host)
  struct TriRef { int prob; int col; int m; };  // col = -1: A itself
  std::vector<TriRef> tri;
  for (int p = 0; p < (int)probs.size(); ++p) {
    const Problem& P = probs[p];
    if (P.n < 1) continue;
    if (!P.lam_in) tri.push_back({p, -1, P.n});
    if (mode != MODE_EIGVALS && P.n >= 2)
      for (int c = 0; c < (int)P.cols.size(); ++c) tri.push_back({p, c, P.n - 1});
  }
  if (tri.empty()) return EEID_OK;

  // ---- device layout: [metadata (uploaded once per call) | data buffers]
  Arena meta, dat;
  std::vector<size_t> lam_off(probs.size(), 0), mu_off(probs.size(), 0), dm_off(probs.size(), 0),
      de_off(probs.size(), 0);
  std::vector<size_t> d_off(tri.size()), e_off(tri.size());
  for (size_t t = 0; t < tri.size(); ++t) {
    d_off[t] = dat.take(sizeof(double) * tri[t].m);
    e_off[t] = dat.take(sizeof(double) * std::max(tri[t].m - 1, 1));
  }
  int max_n = 1;
  for (size_t p = 0; p < probs.size(); ++p) {
    const Problem& P = probs[p];
    max_n = std::max(max_n, P.n);
    if (P.n < 1) continue;
    lam_off[p] = (P.lam_user || P.lam_in) ? SIZE_MAX : dat.take(sizeof(double) * P.n);
    if (mode != MODE_EIGVALS && P.n >= 2)
      mu_off[p] = (mode == MODE_MINORS) ? SIZE_MAX
                                        : dat.take(sizeof(double) * P.cols.size() * (P.n - 1));
    if (mode == MODE_COMPONENTS) {
      dm_off[p] = dat.take(sizeof(double) * P.n);
      de_off[p] = dat.take(sizeof(int) * P.n);
    }
  }
  // tridiagonalisation groups (one persistent launch per configuration)
  std::vector<std::vector<int>> groups(128);
  for (size_t t = 0; t < tri.size(); ++t)
    groups[cfg_key(probs[tri[t].prob].herm ? herm_cfg(tri[t].m) : tri_cfg(ctx, tri[t].m))]
        .push_back((int)t);
  struct GroupPlan { TriCfg cfg; int max_m; int grid; int nchunks; size_t task_off, counter_off,
                     work_off; size_t slot; std::vector<int> idx; int csize = 0; int gsize = 0;
                     size_t gsync_off = 0, gw_off = 0; };
  std::vector<GroupPlan> gplans;
  for (int key = 0; key < 128; ++key) {
    if (groups[key].empty()) continue;
    GroupPlan g;
    g.idx = groups[key];
    std::stable_sort(g.idx.begin(), g.idx.end(),
                     [&](int a, int b) { return tri[a].m > tri[b].m; });  // cost-sorted
    g.max_m = tri[g.idx[0]].m;
    g.cfg = key >= 96 ? herm_cfg(g.max_m) : tri_cfg(ctx, g.max_m);
    const int sms_used = std::max(1, ctx->sms - ctx->sm_reserve);
    // a narrow global build only for a wave that fills the SMs with it (narrow_build_fills)
    if (!g.cfg.smem && !g.cfg.herm && g.cfg.warps < 4 &&
        !narrow_build_fills((int64_t)g.idx.size(), sms_used, blocks_per_sm(ctx, g.cfg, g.max_m)))
      g.cfg = TriCfg{false, 4};
    const int bps = blocks_per_sm(ctx, g.cfg, g.max_m);
    g.grid = (int)std::min<int64_t>((int64_t)g.idx.size(), (int64_t)sms_used * bps);
    // Round launches (serving) of a large group: rounds of two 8-warp CTAs per SM when
    // they finish the group sooner than rounds of one wide CTA per SM (a pair-round takes
    // kRound8x2Per16 single rounds for twice the matrices), as in the plain path's
    // hybrid rounds.  Bitwise the same results.
    if (ctx->round_launches && ctx->overlap_enabled && !g.cfg.smem && !g.cfg.herm &&
        g.cfg.warps >= 12 && bps == 1 && g.grid == sms_used && !rule_covers(ctx, g.max_m) &&
        cfg_supported(1, 8, g.max_m)) {
      const TriCfg c8{false, 8};
      const int b8 = blocks_per_sm(ctx, c8, g.max_m);
      const int nt = (int)g.idx.size(), g8 = sms_used * b8;
      const double t_pairs = (double)((nt + g8 - 1) / g8) * kRound8x2Per16;
      const double t_single = (double)((nt + g.grid - 1) / g.grid);
      if (b8 >= 2 && nt > g.grid && t_pairs < t_single) {
        g.cfg = c8;
        g.grid = g8;
      }
    }
    g.slot = g.cfg.herm ? tridiag_herm_slot_doubles(g.max_m)
             : g.cfg.smem ? 0 : tridiag_global_slot_doubles(g.max_m);
    g.work_off = 0;  // assigned after the rest of the layout (see below)
    g.task_off = meta.take(sizeof(TridiagTask) * g.idx.size());
    g.nchunks = ctx->round_launches ? (int)((g.idx.size() + g.grid - 1) / g.grid) : 1;
    g.counter_off = meta.take(sizeof(int) * g.nchunks);
    gplans.push_back(std::move(g));
  }
  // Cluster plan: a single group of few large reductions runs one cluster of csize CTAs
  // per matrix (one round; each cluster works in one global slot).  Results are
  // bitwise those of the one-CTA global variant.
  if (ctx->clusters_enabled && !ctx->round_launches && gplans.size() == 1 &&
      !gplans[0].cfg.smem && !gplans[0].cfg.herm && !rule_covers(ctx, gplans[0].max_m)) {
    GroupPlan& g = gplans[0];
    const int nt = (int)g.idx.size();
    int c = cluster_size_for(nt, std::max(1, ctx->sms - ctx->sm_reserve), g.max_m);
    const int w = cluster_warps(g.max_m);
    while (c >= 2 && w && tridiag_max_active_clusters(w, c, g.max_m) < nt) c /= 2;
    // the fewest, largest reductions: groups of more CTAs than a cluster can hold
    const int gsz = ctx->groups_enabled
                        ? group_size_for(nt, std::max(1, ctx->sms - ctx->sm_reserve), g.max_m) : 0;
    if (gsz && (w == 12 || w == 16) && tridiag_group_blocks_per_sm(w, g.max_m) >= 1) {
      g.gsize = gsz;
      g.cfg = {false, w};
      g.grid = nt;   // groups (= slots)
      g.gsync_off = meta.take(sizeof(unsigned) * kGroupSyncWords * nt);
    } else if (c >= 2 && w) {
      g.csize = c;
      g.cfg = {false, w};
      g.grid = nt;   // clusters (= slots)
    }
  }
  // Tail overlap.  One group of near-equal tasks (sizes within 1) in more than one
  // round leaves grid - r CTAs idle through its last round (r = tasks mod grid).  Then
  // the first tail_at tasks (whole rounds, every A among them) form the first launch;
  // the last r run as a second launch on the context's greatest-priority stream, and
  // meanwhile the caller's stream bisects A and the minors of the first launch on the
  // SMs the tail leaves free.  Per-task arithmetic is unchanged.
  //
  // Hybrid rounds.  When such a group runs one 16-warp CTA per SM by default and the
  // 8-warp variant fits two CTAs per SM, whole rounds of the 8-warp pair are faster
  // (kRound8x2Per16 < 2); the group then runs its whole pair-rounds that way and a
  // tail of at most one round as the 16-warp second launch.  Both variants give
  // bitwise the same (d, e), so the plan never shows in the results.
  int tail_at = 0, tail_grid = 0, tail_grid_of = 0;
  TriCfg tail_cfg{false, 0};
  int tail_csize = 0;   // the tail launch's cluster size (0: one CTA per matrix)
  size_t counter2_off = 0;
  std::vector<char> in_tail(tri.size(), 0);
  if (ctx->overlap_enabled && !ctx->round_launches && gplans.size() == 1 && mode != MODE_EIGVALS &&
      gplans[0].csize == 0 && gplans[0].gsize == 0 && !gplans[0].cfg.herm) {
    GroupPlan& g = gplans[0];
    const int nt = (int)g.idx.size();
    const bool uniform = tri[g.idx.back()].m + 1 >= tri[g.idx.front()].m;
    auto split_at = [&](int at, int grid) {
      tail_at = at;
      tail_grid = grid;
      tail_grid_of = g.grid;
      counter2_off = meta.take(sizeof(int));
      for (int q = at; q < nt; ++q) in_tail[g.idx[q]] = 1;
    };
    int last_a = -1;
    for (int q = 0; q < nt; ++q)
      if (tri[g.idx[q]].col < 0) last_a = q;
    const TriCfg c8{false, 8};
    const bool wide = !g.cfg.smem && g.cfg.warps >= 12;
    const int blocks8 = (wide && !rule_covers(ctx, g.max_m) && cfg_supported(1, 8, g.max_m))
                            ? blocks_per_sm(ctx, c8, g.max_m) : 0;
    const RoundPlan rp = plan_rounds(nt, g.grid, ctx->sms, wide, blocks8, uniform, last_a);
    tail_cfg = g.cfg;   // the tail runs the group's default variant
    // Cluster rounds instead, when the estimate says they keep the SMs busier than the
    // one-CTA plan (see plan_cluster_rounds).  Same bitwise results either way.
    ClusterRounds cr;
    if (ctx->clusters_enabled && uniform && !g.cfg.smem && !rule_covers(ctx, g.max_m) &&
        g.grid == ctx->sms && 2 * nt > ctx->sms) {
      const int w = g.cfg.warps;
      int active[4];
      for (int k = 0; k < 4; ++k) active[k] = tridiag_max_active_clusters(w, 2 << k, g.max_m);
      double t_single;
      if (rp.hybrid) {
        const int bulk = rp.tail_at > 0 ? rp.tail_at : nt;
        t_single = (double)(bulk / rp.bulk_grid) * kRound8x2Per16 + (rp.tail_at > 0 ? 1.0 : 0.0);
      } else {
        t_single = (double)((nt + g.grid - 1) / g.grid);
      }
      cr = plan_cluster_rounds(nt, ctx->sms, g.max_m, active, t_single);
      if (cr.c1 && last_a >= cr.bulk) cr = ClusterRounds();
    }
    if (cr.c1) {
      g.csize = cr.c1;
      g.grid = cr.per_round;   // clusters (= slots)
      if (cr.bulk < nt) {
        split_at(cr.bulk, nt - cr.bulk);
        tail_csize = cr.c2;
      }
    } else {
      if (rp.hybrid) {
        g.cfg = c8;
        g.grid = rp.bulk_grid;
      }
      if (rp.tail_at > 0) split_at(rp.tail_at, rp.tail_grid);
    }
  }
  // bisection tasks: A's first (their eigenvalues seed the minors' brackets); with the
  // tail overlap the minors of the tail are bisected in a second launch
  std::vector<int> bis_a, bis_m, bis_m2;
  for (size_t t = 0; t < tri.size(); ++t)
    (tri[t].col < 0 ? bis_a : in_tail[t] ? bis_m2 : bis_m).push_back((int)t);
  const size_t bt_off = meta.take(sizeof(BisectTask) * tri.size());
  // Bisection blocks, largest tasks first.  Runs of consecutive tasks (the minors of one
  // matrix) of one small size m share a block, threads / m of them at a time.  A launch
  // with few eigenvalues (fewer than 128 per SM) uses 64-lane blocks so that it spreads
  // over more SMs (a single large matrix: the latency of a few-component call).
  auto eig_count = [&](const std::vector<int>& ts) {
    int64_t c = 0;
    for (int t : ts) c += tri[t].m;
    return c;
  };
  const int bis_threads_a = eig_count(bis_a) <= (int64_t)ctx->sms * 128 ? 64 : kBisectThreads;
  const int bis_threads_m =
      eig_count(bis_m) + eig_count(bis_m2) <= (int64_t)ctx->sms * 128 ? 64 : kBisectThreads;
  auto items_of = [&](const std::vector<int>& ts, std::vector<BisectItem>& items, int& mm,
                      int threads) {
    std::vector<int> order = ts;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tri[a].m > tri[b].m; });
    mm = 1;
    for (int t : order) mm = std::max(mm, tri[t].m);
    std::vector<BisectBlock> blocks;
    plan_bisect_blocks(order, [&](int t) { return tri[t].m; }, threads, kBisectMaxPack, blocks);
    for (const BisectBlock& b : blocks) {
      BisectItem it;
      it.task = b.task;
      it.k0 = b.k0;
      it.ntask = b.ntask;
      items.push_back(it);
    }
  };
  std::vector<BisectItem> items_a, items_m, items_m2;
  int mm_a = 1, mm_m = 1, mm_m2 = 1;
  items_of(bis_a, items_a, mm_a, bis_threads_a);
  items_of(bis_m, items_m, mm_m, bis_threads_m);
  items_of(bis_m2, items_m2, mm_m2, bis_threads_m);
  const size_t bia_off = meta.take(sizeof(BisectItem) * std::max<size_t>(items_a.size(), 1));
  // the minors' items, then the tail minors' items, in one array (one launch over both
  // when the tail is not split off)
  const size_t bim_off =
      meta.take(sizeof(BisectItem) * std::max<size_t>(items_m.size() + items_m2.size(), 1));
  const size_t bim2_off = bim_off + sizeof(BisectItem) * items_m.size();
  // identity
  std::vector<IdentityItem> iitems;
  std::vector<DenomItem> ditems;
  size_t dt_off = 0, ip_off = 0, ii_off = 0, di_off = 0;
  std::vector<size_t> rows_off(probs.size(), 0);
  if (mode == MODE_COMPONENTS) {
    for (size_t p = 0; p < probs.size(); ++p)
      if (probs[p].n >= 1)
        rows_off[p] = meta.take(sizeof(int) * std::max<size_t>(probs[p].rows.size(), 1));
    dt_off = meta.take(sizeof(DenomTask) * probs.size());
    ip_off = meta.take(sizeof(IdentityProblem) * probs.size());
    for (size_t p = 0; p < probs.size(); ++p)
      if (probs[p].n >= 1)
        for (int r0 = 0; r0 < (int)probs[p].rows.size(); r0 += kDenomThreads)
          ditems.push_back({(int)p, r0});
    di_off = meta.take(sizeof(DenomItem) * std::max<size_t>(ditems.size(), 1));
    for (size_t p = 0; p < probs.size(); ++p) {
      const Problem& P = probs[p];
      if (P.n < 1) continue;
      for (int c = 0; c < (int)P.cols.size(); ++c)
        for (int r0 = 0; r0 < (int)P.rows.size(); r0 += kIdentityThreads)
          iitems.push_back({(int)p, c, r0});
    }
    ii_off = meta.take(sizeof(IdentityItem) * std::max<size_t>(iitems.size(), 1));
  }
  const size_t meta_bytes = meta.off;
  // Working slots of the global-memory groups go last.  If the whole layout would
  // exceed the context's budget, fewer persistent CTAs (slots) are used: the same
  // tasks in more rounds, with identical per-task arithmetic.
  {
    size_t slots_total = 0;
    for (auto& g : gplans) slots_total += sizeof(double) * g.slot * g.grid;
    const size_t fixed = meta_bytes + dat.off + kAlign * (gplans.size() + 1);
    if (slots_total > 0 && fixed + slots_total > ctx->budget) {
      if (fixed >= ctx->budget)
        return fail(EEID_ERR_NOMEM, "task data of %zu bytes exceeds the HBM budget of %zu bytes",
                    fixed, ctx->budget);
      const double scale = (double)(ctx->budget - fixed) / (double)slots_total;
      for (auto& g : gplans) {
        if (g.cfg.smem) continue;
        if (g.csize || g.gsize) {   // fewer slots than matrices: back to one CTA per matrix
          g.csize = 0;
          g.gsize = 0;
          g.cfg = tri_cfg(ctx, g.max_m);
          g.slot = tridiag_global_slot_doubles(g.max_m);
          g.grid = std::min<int>((int)g.idx.size(), ctx->sms * blocks_per_sm(ctx, g.cfg, g.max_m));
        }
        const int ng = (int)((double)g.grid * scale);
        if (ng < 1)
          return fail(EEID_ERR_NOMEM, "one working slot (%zu bytes) does not fit the HBM budget",
                      sizeof(double) * g.slot);
        g.grid = ng;
      }
    }
    for (auto& g : gplans) {
      if (!g.cfg.smem) g.work_off = dat.take(sizeof(double) * g.slot * g.grid);
      if (g.gsize)
        g.gw_off = dat.take(sizeof(double) * (size_t)(g.max_m + 96) * g.grid);
    }
    // fewer slots than planned: the tail would not be a round of them, so the group
    // runs as one launch (both minor bisections then follow it)
    if (tail_at > 0 && gplans[0].grid != tail_grid_of) tail_at = 0;
  }
  eeid_status st = ensure_ws(ctx, meta_bytes + dat.off);
  if (st != EEID_OK) return st;
  if (tail_at > 0) {
    st = ensure_aux(ctx);
    if (st != EEID_OK) return st;
  }
  char* ws = ctx->ws;
  char* wd = ws + meta_bytes;
  auto D = [&](size_t off) { return (double*)(wd + off); };

  // ---- host image of the metadata region (counters stay zero)
  char* img = nullptr;
  if (ge) {
    EEID_CK(cudaMallocHost((void**)&ge->pinned, std::max<size_t>(meta_bytes, 256)),
            "cudaMallocHost(graph metadata)");
    img = ge->pinned;
  } else {
    st = ensure_stage(ctx, meta_bytes);
    if (st != EEID_OK) return st;
    img = ctx->h_stage;
  }
  memset(img, 0, meta_bytes);
  auto lam_ptr = [&](int p) {
    return probs[p].lam_in ? const_cast<double*>(probs[p].lam_in)
                           : probs[p].lam_user ? probs[p].lam_user : D(lam_off[p]);
  };
  auto mu_ptr = [&](int p) {
    return mode == MODE_MINORS ? probs[p].mu_user : D(mu_off[p]);
  };
  for (auto& g : gplans) {
    TridiagTask* tt = (TridiagTask*)(img + g.task_off);
    for (size_t q = 0; q < g.idx.size(); ++q) {
      const TriRef& r = tri[g.idx[q]];
      const Problem& P = probs[r.prob];
      tt[q] = {P.dA, P.lda, P.n, r.col < 0 ? -1 : P.cols[r.col], D(d_off[g.idx[q]]),
               D(e_off[g.idx[q]]), r.col < 0 ? -1 : P.rot, 0};
    }
  }
  {
    BisectTask* bt = (BisectTask*)(img + bt_off);
    for (size_t t = 0; t < tri.size(); ++t) {
      const TriRef& r = tri[t];
      double* eig = (r.col < 0) ? lam_ptr(r.prob) : mu_ptr(r.prob) + (size_t)r.col * (r.m);
      bt[t] = {D(d_off[t]), D(e_off[t]), r.m, r.col < 0 ? nullptr : lam_ptr(r.prob), eig};
    }
    if (!items_a.empty()) memcpy(img + bia_off, items_a.data(), sizeof(BisectItem) * items_a.size());
    if (!items_m.empty()) memcpy(img + bim_off, items_m.data(), sizeof(BisectItem) * items_m.size());
    if (!items_m2.empty())
      memcpy(img + bim2_off, items_m2.data(), sizeof(BisectItem) * items_m2.size());
    if (tail_at == 0) {   // tail dropped by the budget fit: one launch over both parts
      items_m.insert(items_m.end(), items_m2.begin(), items_m2.end());
      items_m2.clear();
      mm_m = std::max(mm_m, mm_m2);
    }
  }
  if (mode == MODE_COMPONENTS) {
    DenomTask* dt = (DenomTask*)(img + dt_off);
    IdentityProblem* ip = (IdentityProblem*)(img + ip_off);
    for (size_t p = 0; p < probs.size(); ++p) {
      const Problem& P = probs[p];
      if (P.n < 1) continue;
      dt[p] = {lam_ptr((int)p), P.n, D(dm_off[p]), (int*)(wd + de_off[p]),
               (const int*)(ws + rows_off[p]), (int)P.rows.size()};
      memcpy(img + rows_off[p], P.rows.data(), sizeof(int) * P.rows.size());
      ip[p] = {lam_ptr((int)p), D(dm_off[p]), (const int*)(wd + de_off[p]),
               P.n >= 2 ? mu_ptr((int)p) : nullptr, (const int*)(ws + rows_off[p]), P.n,
               (int)P.rows.size(), (int)P.cols.size(), P.out};
    }
    if (!iitems.empty()) memcpy(img + ii_off, iitems.data(), sizeof(IdentityItem) * iitems.size());
    if (!ditems.empty()) memcpy(img + di_off, ditems.data(), sizeof(DenomItem) * ditems.size());
  }
  auto enqueue_launches = [&]() -> eeid_status {
  // ---- launches (optionally bracketed by per-phase events)
  for (int ph = 0; ph < EEID_NUM_PHASES; ++ph) ctx->ran[ph] = false;
  auto mark = [&](int ph, int which, cudaStream_t on) -> cudaError_t {
    if (!ctx->timing) return cudaSuccess;
    if (which == 1) ctx->ran[ph] = true;
    // inside a capture the record must become a graph node (external event)
    return ge ? cudaEventRecordWithFlags(ctx->ev[ph][which], on, cudaEventRecordExternal)
              : cudaEventRecord(ctx->ev[ph][which], on);
  };
  EEID_CK(mark(EEID_PHASE_TRIDIAG, 0, stream), "event");
  for (auto& g : gplans) {
    TridiagLaunch L;
    L.tasks = (const TridiagTask*)(ws + g.task_off);
    L.ntasks = tail_at > 0 ? tail_at : (int)g.idx.size();
    L.counter = (int*)(ws + g.counter_off);
    L.work = g.cfg.smem ? nullptr : D(g.work_off);
    L.work_stride = (int64_t)g.slot;
    L.max_m = g.max_m;
    L.status = status_word;
    auto launch_group = [&](int grid, const TridiagLaunch& LL, cudaStream_t on) {
      return g.cfg.herm ? launch_tridiag_herm(g.cfg.warps, grid, LL, on)
                        : launch_tridiag(g.cfg.smem, g.cfg.warps, grid, LL, on, g.cfg.hi);
    };
    if (g.nchunks > 1) {
      // round launches: chunk c takes tasks [c*chunk, ...) with its own counter.  When the
      // last round would be short (at most half the SMs' worth of matrices), the whole
      // rounds are launched full and that remainder runs as one launch of clusters.
      const int total = L.ntasks;
      int chunk = (total + g.nchunks - 1) / g.nchunks, last_c = 0, last_w = 0;
      if (ctx->clusters_enabled && !g.cfg.smem && !g.cfg.herm && !rule_covers(ctx, g.max_m)) {
        const int rem = total % g.grid;
        const int sms_used = std::max(1, ctx->sms - ctx->sm_reserve);
        const int w = cluster_warps(g.max_m);
        int c = rem > 0 && w ? cluster_size_for(rem, sms_used, g.max_m) : 0;
        while (c >= 2 && tridiag_max_active_clusters(w, c, g.max_m) < rem) c /= 2;
        if (c >= 2) {
          chunk = g.grid;
          last_c = c;
          last_w = w;
        }
      }
      const TridiagTask* t0 = L.tasks;
      for (int c = 0; c < g.nchunks; ++c) {
        const int a = c * chunk, b = std::min(total, a + chunk);
        if (a >= b) break;
        L.tasks = t0 + a;
        L.ntasks = b - a;
        L.counter = (int*)(ws + g.counter_off) + c;
        if (last_c && b - a < chunk)
          EEID_CK(launch_tridiag_cluster(last_w, b - a, last_c, L, stream),
                  "tridiag cluster launch");
        else
          EEID_CK(launch_group(std::min(g.grid, b - a), L, stream), "tridiag launch");
        ctx->launches++;
      }
      continue;
    }
    if (g.gsize) {
      L.group = g.gsize;
      L.gsync = (unsigned*)(ws + g.gsync_off);
      L.gw = D(g.gw_off);
      EEID_CK(launch_tridiag_group(g.cfg.warps, g.grid, g.gsize, L, stream),
              "tridiag group launch");
    } else if (g.csize) {
      EEID_CK(launch_tridiag_cluster(g.cfg.warps, g.grid, g.csize, L, stream),
              "tridiag cluster launch");
    } else {
      EEID_CK(launch_group(g.grid, L, stream), "tridiag launch");
    }
    ctx->launches++;
    if (tail_at > 0) {
      // the tail: same slots (the first launch is done with them), its own counter
      EEID_CK(cudaEventRecord(ctx->fork_ev, stream), "fork record");
      EEID_CK(cudaStreamWaitEvent(ctx->aux_stream, ctx->fork_ev, 0), "fork wait");
      L.tasks += tail_at;
      L.ntasks = (int)g.idx.size() - tail_at;
      L.counter = (int*)(ws + counter2_off);
      if (tail_csize)
        EEID_CK(launch_tridiag_cluster(tail_cfg.warps, tail_grid, tail_csize, L, ctx->aux_stream),
                "tridiag tail cluster launch");
      else
        EEID_CK(launch_tridiag(tail_cfg.smem, tail_cfg.warps, tail_grid, L, ctx->aux_stream),
                "tridiag tail launch");
      ctx->launches++;
    }
  }
  if (tail_at > 0) {
    EEID_CK(mark(EEID_PHASE_TRIDIAG, 1, ctx->aux_stream), "event");
    EEID_CK(cudaEventRecord(ctx->join_ev, ctx->aux_stream), "join record");
  } else {
    EEID_CK(mark(EEID_PHASE_TRIDIAG, 1, stream), "event");
  }
  const BisectTask* btd = (const BisectTask*)(ws + bt_off);
  if (!items_a.empty()) {
    EEID_CK(mark(EEID_PHASE_BISECT_A, 0, stream), "event");
    EEID_CK(launch_bisect(btd, (const BisectItem*)(ws + bia_off), (int)items_a.size(), mm_a,
                          status_word, stream, bis_threads_a), "bisect(A) launch");
    ctx->launches++;
    EEID_CK(mark(EEID_PHASE_BISECT_A, 1, stream), "event");
  }
  if (mode == MODE_COMPONENTS) {
    EEID_CK(mark(EEID_PHASE_DENOMINATORS, 0, stream), "event");
    EEID_CK(launch_denominators((const DenomTask*)(ws + dt_off), (const DenomItem*)(ws + di_off),
                                (int)ditems.size(), max_n,
                                status_word, stream), "denominators launch");
    ctx->launches++;
    EEID_CK(mark(EEID_PHASE_DENOMINATORS, 1, stream), "event");
  }
  if (!items_m.empty() || !items_m2.empty()) {
    EEID_CK(mark(EEID_PHASE_BISECT_MINORS, 0, stream), "event");
    if (!items_m.empty()) {
      EEID_CK(launch_bisect(btd, (const BisectItem*)(ws + bim_off), (int)items_m.size(), mm_m,
                            status_word, stream, bis_threads_m), "bisect(minors) launch");
      ctx->launches++;
    }
    if (tail_at > 0) EEID_CK(cudaStreamWaitEvent(stream, ctx->join_ev, 0), "join wait");
    if (!items_m2.empty()) {
      EEID_CK(launch_bisect(btd, (const BisectItem*)(ws + bim2_off), (int)items_m2.size(), mm_m2,
                            status_word, stream, bis_threads_m), "bisect(tail minors) launch");
      ctx->launches++;
    }
    EEID_CK(mark(EEID_PHASE_BISECT_MINORS, 1, stream), "event");
  } else if (tail_at > 0) {
    EEID_CK(cudaStreamWaitEvent(stream, ctx->join_ev, 0), "join wait");
  }
  if (mode == MODE_COMPONENTS && !iitems.empty()) {
    EEID_CK(mark(EEID_PHASE_IDENTITY, 0, stream), "event");
    EEID_CK(launch_identity((const IdentityProblem*)(ws + ip_off),
                            (const IdentityItem*)(ws + ii_off), (int)iitems.size(), max_n, stream),
            "identity launch");
    ctx->launches++;
    EEID_CK(mark(EEID_PHASE_IDENTITY, 1, stream), "event");
  }
    return EEID_OK;
  };
  const cudaStream_t user_stream = stream;
  const int64_t launches_before = ctx->launches;
  if (ge) {
    stream = ctx->cap_stream;
    EEID_CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  }
  EEID_CK(cudaMemcpyAsync(ws, img, meta_bytes, cudaMemcpyHostToDevice, stream),
          "cudaMemcpyAsync(metadata)");
  if (!ge) {
    EEID_CK(cudaEventRecord(ctx->stage_ev, stream), "cudaEventRecord(stage)");
    ctx->stage_used = true;
  }
  eeid_status lst = enqueue_launches();
  if (ge) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(stream, &graph);
    if (lst != EEID_OK) {
      if (graph) cudaGraphDestroy(graph);
      return lst;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    // node priorities keep the tail launch ahead of the overlapping bisection
    e = cudaGraphInstantiate(&ge->exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    ge->nkernels = (int)(ctx->launches - launches_before);
    ctx->launches = launches_before;  // counted when the graph is launched
    (void)user_stream;
  }
  return lst;
}


}  // namespace

// ===================================================================== C ABI
extern "C" {

const char* eeid_last_error(void) { return g_err.c_str(); }

eeid_status eeid_ctx_create(int device, size_t hbm_budget_bytes, eeid_ctx** out) {
  if (!out) return fail(EEID_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(EEID_ERR_CUDA, "no CUDA device available (%s)",
                e != cudaSuccess ? cudaGetErrorString(e) : "count is 0");
  }
  if (device < 0 || device >= ndev) return fail(EEID_ERR_INVALID, "device %d out of range", device);
  EEID_CK(cudaSetDevice(device), "cudaSetDevice");
  cudaDeviceProp prop;
  EEID_CK(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
  size_t fr = 0, tot = 0;
  EEID_CK(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
  eeid_ctx* c = new eeid_ctx();
  c->device = device;
  c->sms = prop.multiProcessorCount;
  c->budget = hbm_budget_bytes ? hbm_budget_bytes : fr / 2;
  e = cudaMalloc((void**)&c->d_status, sizeof(unsigned) * kStatusSlots);
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(unsigned) * kStatusSlots);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_status, sizeof(unsigned) * kStatusSlots);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming);
  // every kernel loaded now, not at its first launch (see preload_tridiag)
  if (e == cudaSuccess) e = preload_tridiag();
  if (e == cudaSuccess) e = preload_bisect();
  if (e == cudaSuccess) e = preload_identity();
  if (e == cudaSuccess) e = preload_vectors();
  if (e == cudaSuccess) e = preload_tridiag_herm();
  if (e != cudaSuccess) {
    eeid_ctx_destroy(c);
    return cuda_fail(e, "context setup");
  }
  *out = c;
  return EEID_OK;
}

void eeid_ctx_destroy(eeid_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  clear_graphs(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->host_call_buf) cudaFree(ctx->host_call_buf);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  if (ctx->stage_ev) cudaEventDestroy(ctx->stage_ev);
  if (ctx->vbuf) cudaFree(ctx->vbuf);
  if (ctx->h_vec) cudaFreeHost(ctx->h_vec);
  if (ctx->vec_ev) cudaEventDestroy(ctx->vec_ev);
  for (int p = 0; p < EEID_NUM_PHASES; ++p)
    for (int w = 0; w < 2; ++w)
      if (ctx->ev[p][w]) cudaEventDestroy(ctx->ev[p][w]);
  delete ctx;
}

int64_t eeid_launch_count(const eeid_ctx* ctx) { return ctx ? ctx->launches : 0; }

int64_t eeid_vector_refs(const eeid_ctx* ctx) { return ctx ? ctx->vec_refs : 0; }

eeid_status eeid_check_barrier_timeout(eeid_ctx* ctx, void* stream) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  EEID_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  // a 2 x 2 matrix for a group of two CTAs, one of them never launched
  const int m = 2;
  const size_t slot = tridiag_global_slot_doubles(m);
  const size_t off_task = 0, off_sync = 256, off_a = 512, off_de = off_a + 64,
               off_gw = off_de + 64, off_slot = off_gw + sizeof(double) * (m + 96);
  const size_t bytes = off_slot + sizeof(double) * slot;
  char* buf = nullptr;
  EEID_CK(cudaMalloc((void**)&buf, bytes), "cudaMalloc(barrier check)");
  const double A[4] = {2.0, 0.0, 1.0, 3.0};
  TridiagTask t{(const double*)(buf + off_a), 2, 2, -1, (double*)(buf + off_de),
                (double*)(buf + off_de) + 2, -1, 0};
  cudaError_t e = cudaMemsetAsync(buf, 0, bytes, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + off_a, A, sizeof(A), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + off_task, &t, sizeof(t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    TridiagLaunch L;
    L.tasks = (const TridiagTask*)(buf + off_task);
    L.ntasks = 1;
    L.counter = nullptr;
    L.work = (double*)(buf + off_slot);
    L.work_stride = (int64_t)slot;
    L.max_m = m;
    L.status = ctx->d_status + status_slot(ctx, s, true);
    L.group = 2;
    L.gsync = (unsigned*)(buf + off_sync);
    L.gw = (double*)(buf + off_gw);
    e = launch_tridiag_group_short(L, s);
    if (e == cudaSuccess) ctx->launches++;
  }
  // the host copies above read stack memory: wait for them (and the launch) before return
  const cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFree(buf);
  EEID_CK(e, "barrier check launch");
  EEID_CK(e2, "barrier check");
  return EEID_OK;
}

eeid_status eeid_tune_tridiag(eeid_ctx* ctx, int m_lo, int m_hi, int path, int warps) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  if (m_lo < 1 || m_hi < m_lo || path < 0 || path > 2)
    return fail(EEID_ERR_INVALID, "bad tuning rule");
  if (!cfg_supported(path, warps, m_hi))
    return fail(EEID_ERR_INVALID, "unsupported variant (path %d, %d warps) for m <= %d", path, warps,
                m_hi);
  ctx->rules.push_back({m_lo, m_hi, path, warps});
  ctx->rules_version++;
  return EEID_OK;
}

eeid_status eeid_autotune(eeid_ctx* ctx, int max_m, const char* cache_path) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  if (max_m < 1) return fail(EEID_ERR_INVALID, "max_m must be >= 1");
  EEID_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaDeviceProp prop;
  EEID_CK(cudaGetDeviceProperties(&prop, ctx->device), "cudaGetDeviceProperties");
  char header[384];
  snprintf(header, sizeof header, "eeid-tune v3 sms=%d name=%s", prop.multiProcessorCount, prop.name);
  const int mmax = std::min(max_m, 1024);
  std::vector<eeid_ctx::Rule> chosen;
  // ---- cached table
  if (cache_path) {
    FILE* f = fopen(cache_path, "r");
    if (f) {
      char line[512];
      bool ok = fgets(line, sizeof line, f) != nullptr;
      if (ok) {
        line[strcspn(line, "\r\n")] = 0;
        ok = strcmp(line, header) == 0;
      }
      int lo, hi, path, w;
      while (ok && fscanf(f, "%d %d %d %d", &lo, &hi, &path, &w) == 4) {
        if (!cfg_supported(path, w, hi) || lo < 1 || hi < lo) { ok = false; break; }
        chosen.push_back({lo, hi, path, w});
      }
      fclose(f);
      if (ok && !chosen.empty() && chosen.back().hi >= mmax) {
        for (auto& r : chosen) ctx->rules.push_back(r);
        ctx->rules_version++;
        return EEID_OK;
      }
      chosen.clear();
    }
  }
  // ---- measure: for each bucket, every supported variant on a wave of minors whose sizes
  // cover the bucket evenly, largest first (as a batch of uneven matrices does), long enough (about
  // 1.5e11 flops, at least two tasks per SM) that the last partial round weighs little
  static const int kBuckets[] = {16, 24, 32, 48, 64, 96, 128, 160, 192, 256, 384, 512, 768, 1024};
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  EEID_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "tune stream");
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
  };
  if (ce != cudaSuccess) { cleanup(); return cuda_fail(ce, "tune events"); }
  int prev = 0;
  for (int bm : kBuckets) {
    if (prev >= mmax) break;
    const int m = std::min(bm, mmax);
    const int n = m + 1;
    const int lo = prev + 1;   // minor sizes lo..m
    double flops_task = 0.0;
    for (int q = lo; q <= m; ++q) flops_task += 4.0 / 3.0 * (double)q * q * q;
    flops_task /= (double)(m - lo + 1);
    const int T = (int)std::max<double>(2.0 * ctx->sms,
                                        std::min<double>(64.0 * ctx->sms, 1.5e11 / flops_task));
    struct Cand { TriCfg c; int grid; size_t slot; };
    std::vector<Cand> cands;
    for (int path = 0; path < 3; ++path)
      for (int w : {1, 2, 4, 8, 16}) {
        if (!cfg_supported(path, w, m)) continue;
        TriCfg c = cfg_of(path, w);
        const int grid = (int)std::min<int64_t>(T, (int64_t)ctx->sms * blocks_per_sm(ctx, c, m));
        cands.push_back({c, grid, c.smem ? 0 : tridiag_global_slot_doubles(m)});
      }
    size_t work_bytes = 0;
    for (auto& c : cands) work_bytes = std::max(work_bytes, sizeof(double) * c.slot * c.grid);
    Arena ar;
    const size_t a_off = ar.take(sizeof(double) * (size_t)n * n);
    const size_t t_off = ar.take(sizeof(TridiagTask) * T);
    const size_t c_off = ar.take(sizeof(int));
    const size_t de_off = ar.take(sizeof(double) * (size_t)T * (2 * m));
    const size_t w_off = ar.take(work_bytes);
    st = ensure_ws(ctx, ar.off);
    if (st != EEID_OK) { cleanup(); return st; }
    char* ws = ctx->ws;
    double* A = (double*)(ws + a_off);
    std::vector<TridiagTask> tasks(T);
    for (int t = 0; t < T; ++t) {
      double* d = (double*)(ws + de_off) + (size_t)t * 2 * m;
      // leading nt x nt block (minor size nt - 1), largest first like a real batch's
      // cost-sorted task list
      const int nt = m + 1 - (int)((int64_t)t * (m - lo + 1) / T);
      tasks[t] = {A, n, nt, t % nt, d, d + m};
    }
    ce = launch_fill_symmetric(A, n, n, 0x5eedULL + (unsigned long long)m, s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(ws + t_off, tasks.data(), sizeof(TridiagTask) * T, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) { cleanup(); return cuda_fail(ce, "tune setup"); }
    float best_ms = 1e30f;
    TriCfg best = tri_cfg_default(m);
    for (auto& c : cands) {
      TridiagLaunch L;
      L.tasks = (const TridiagTask*)(ws + t_off);
      L.ntasks = T;
      L.counter = (int*)(ws + c_off);
      L.work = (double*)(ws + w_off);
      L.work_stride = (int64_t)c.slot;
      L.max_m = m;
      L.status = ctx->d_status;
      float msr = 0.f;
      for (int rep = 0; rep < 2 && ce == cudaSuccess; ++rep) {
        ce = cudaMemsetAsync(ws + c_off, 0, sizeof(int), s);
        if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
        if (ce == cudaSuccess) ce = launch_tridiag(c.c.smem, c.c.warps, c.grid, L, s, c.c.hi);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&msr, e0, e1);
      }
      if (ce != cudaSuccess) { cleanup(); return cuda_fail(ce, "tune run"); }
      if (msr < best_ms) { best_ms = msr; best = c.c; }
    }
    chosen.push_back({prev + 1, m, path_of(best), best.warps});
    prev = m;
  }
  cleanup();
  for (auto& r : chosen) ctx->rules.push_back(r);
  ctx->rules_version++;
  if (cache_path) {
    FILE* f = fopen(cache_path, "w");
    if (f) {
      fprintf(f, "%s\n", header);
      for (auto& r : chosen) fprintf(f, "%d %d %d %d\n", r.lo, r.hi, r.path, r.warps);
      fclose(f);
    }
  }
  return EEID_OK;
}

eeid_status eeid_set_graphs(eeid_ctx* ctx, int enable) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  ctx->graphs_enabled = enable != 0;
  if (!ctx->graphs_enabled) {
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    clear_graphs(ctx);
  }
  return EEID_OK;
}

}  // extern "C"

namespace eeid {
eeid_status set_round_launches(eeid_ctx* ctx, int enable) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  ctx->round_launches = enable != 0;
  return EEID_OK;
}

eeid_status reserve_workspace(eeid_ctx* ctx, size_t device_bytes, size_t staging_bytes) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  EEID_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  st = ensure_ws(ctx, std::min(device_bytes, ctx->budget));
  if (st == EEID_OK) st = ensure_stage(ctx, staging_bytes);
  return st;
}

eeid_status set_sm_reserve(eeid_ctx* ctx, int sms) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  ctx->sm_reserve = std::max(0, std::min(sms, ctx->sms - 1));
  return EEID_OK;
}
}  // namespace eeid

extern "C" {

eeid_status eeid_set_clusters(eeid_ctx* ctx, int mode) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  if (mode < 0 || mode > 2) return fail(EEID_ERR_INVALID, "cluster mode %d (0, 1 or 2)", mode);
  ctx->clusters_enabled = mode != 0;   // part of the graph key: no graph goes stale
  ctx->groups_enabled = mode == 2;
  return EEID_OK;
}

eeid_status eeid_set_overlap(eeid_ctx* ctx, int enable) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  ctx->overlap_enabled = enable != 0;   // part of the graph key: no graph goes stale
  return EEID_OK;
}

eeid_status eeid_tune_reset(eeid_ctx* ctx) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  ctx->rules.clear();
  ctx->rules_version++;
  return EEID_OK;
}

eeid_status eeid_set_timing(eeid_ctx* ctx, int enable) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  EEID_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (enable && !ctx->ev[0][0]) {
    for (int p = 0; p < EEID_NUM_PHASES; ++p)
      for (int w = 0; w < 2; ++w) EEID_CK(cudaEventCreate(&ctx->ev[p][w]), "cudaEventCreate");
  }
  ctx->timing = enable != 0;
  return EEID_OK;
}

int eeid_phase_times(eeid_ctx* ctx, double* ms, int cap) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  if (!ms || cap < 0) return fail(EEID_ERR_INVALID, "bad output array");
  if (!ctx->ev[0][0]) return fail(EEID_ERR_INVALID, "timing was never enabled");
  EEID_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  const int n = cap < EEID_NUM_PHASES ? cap : EEID_NUM_PHASES;
  for (int p = 0; p < n; ++p) {
    ms[p] = 0.0;
    if (!ctx->ran[p]) continue;
    EEID_CK(cudaEventSynchronize(ctx->ev[p][1]), "cudaEventSynchronize");
    float t = 0.f;
    EEID_CK(cudaEventElapsedTime(&t, ctx->ev[p][0], ctx->ev[p][1]), "cudaEventElapsedTime");
    ms[p] = t;
  }
  return n;
}

eeid_status eeid_sync(eeid_ctx* ctx, void* stream) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  EEID_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  // a stream this context never ran on, or one beyond the table, has the shared word
  const int slot = status_slot(ctx, s, false);
  // read and clear this stream's word in its own order, then wait for the stream
  EEID_CK(cudaMemcpyAsync(ctx->h_status + slot, ctx->d_status + slot, sizeof(unsigned),
                          cudaMemcpyDeviceToHost, s), "status read");
  EEID_CK(cudaMemsetAsync(ctx->d_status + slot, 0, sizeof(unsigned), s), "status clear");
  EEID_CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  const unsigned bits = ctx->h_status[slot];
  if (bits & ST_BAD_TASK) return fail(EEID_ERR_INVALID, "a kernel met a task beyond its size limit");
  if (bits & ST_TIMEOUT)
    return fail(EEID_ERR_TIMEOUT, "a cooperative reduction's barrier wait ran out; its outputs are invalid");
  if (bits & ST_DEGENERATE)
    return fail(EEID_WARN_DEGENERATE, "equal eigenvalues of A: Eq. 1 is 0/0; rows set to NaN");
  if (bits & ST_SMALL_GAP)
    return fail(EEID_WARN_SMALL_GAP, "minimum relative eigenvalue gap below 1e-4");
  return EEID_OK;
}

eeid_status eeid_eigvals(eeid_ctx* ctx, const double* dA, int64_t lda, int64_t n, double* d_lambda,
                         void* stream) {
  eeid_status st = check_ctx(ctx);
  if (st == EEID_OK) st = check_matrix(dA, lda, n);
  if (st != EEID_OK) return st;
  if (n == 0) return EEID_OK;
  if (!d_lambda) return fail(EEID_ERR_INVALID, "d_lambda is NULL");
  std::vector<Problem> probs(1);
  probs[0] = {dA, lda, (int)n, {}, {}, nullptr, d_lambda, nullptr};
  return run(ctx, probs, MODE_EIGVALS, (cudaStream_t)stream);
}

eeid_status eeid_minor_eigvals(eeid_ctx* ctx, const double* dA, int64_t lda, int64_t n,
                               const int64_t* h_cols, int64_t ncols, double* d_mu, void* stream) {
  eeid_status st = check_ctx(ctx);
  if (st == EEID_OK) st = check_matrix(dA, lda, n);
  if (st != EEID_OK) return st;
  std::vector<Problem> probs(1);
  st = parse_indices(h_cols, ncols, n, "cols", probs[0].cols);
  if (st != EEID_OK) return st;
  if (ncols == 0 || n <= 1) return EEID_OK;
  if (!d_mu) return fail(EEID_ERR_INVALID, "d_mu is NULL");
  probs[0].dA = dA; probs[0].lda = lda; probs[0].n = (int)n;
  probs[0].out = nullptr; probs[0].lam_user = nullptr; probs[0].mu_user = d_mu;
  return run(ctx, probs, MODE_MINORS, (cudaStream_t)stream);
}

static eeid_status make_component_problem(const double* dA, int64_t lda, int64_t n,
                                          const int64_t* h_rows, int64_t nrows,
                                          const int64_t* h_cols, int64_t ncols, double* d_out,
                                          double* d_lambda_opt, Problem& P) {
  eeid_status st = check_matrix(dA, lda, n);
  if (st != EEID_OK) return st;
  st = parse_indices(h_rows, nrows, n, "rows", P.rows);
  if (st != EEID_OK) return st;
  st = parse_indices(h_cols, ncols, n, "cols", P.cols);
  if (st != EEID_OK) return st;
  if (nrows > 0 && ncols > 0 && !d_out) return fail(EEID_ERR_INVALID, "d_out is NULL");
  P.dA = dA; P.lda = lda; P.n = (int)n; P.out = d_out; P.lam_user = d_lambda_opt; P.mu_user = nullptr;
  P.all_rows = (h_rows == nullptr);
  P.all_cols = (h_cols == nullptr);
  if (nrows == 0 || ncols == 0) P.n = 0;  // no-op problem
  return EEID_OK;
}

eeid_status eeid_components(eeid_ctx* ctx, const double* dA, int64_t lda, int64_t n,
                            const int64_t* h_rows, int64_t nrows, const int64_t* h_cols,
                            int64_t ncols, double* d_out, double* d_lambda_opt, void* stream) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  std::vector<Problem> probs(1);
  st = make_component_problem(dA, lda, n, h_rows, nrows, h_cols, ncols, d_out, d_lambda_opt,
                              probs[0]);
  if (st != EEID_OK) return st;
  if (probs[0].n == 0) return EEID_OK;
  return run(ctx, probs, MODE_COMPONENTS, (cudaStream_t)stream);
}

eeid_status eeid_components_batched(eeid_ctx* ctx, const eeid_problem* in, int64_t count,
                                    void* stream) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  if (count < 0 || (count > 0 && !in)) return fail(EEID_ERR_INVALID, "bad problem array");
  std::vector<Problem> probs(count);
  for (int64_t p = 0; p < count; ++p) {
    st = make_component_problem(in[p].dA, in[p].lda, in[p].n, in[p].h_rows, in[p].nrows,
                                in[p].h_cols, in[p].ncols, in[p].d_out, in[p].d_lambda, probs[p]);
    if (st != EEID_OK) {
      g_err = "problem " + std::to_string(p) + ": " + g_err;
      return st;
    }
  }
  // Replay the captured graph of an identical earlier batch, or capture a new one.
  EEID_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  if (!ctx->graphs_enabled) return run(ctx, probs, MODE_COMPONENTS, s);
  // the graph bakes in the status word of the stream it was captured for
  const int slot = status_slot(ctx, s, true);
  std::string key = std::to_string(slot) + ":" + batch_key(probs, ctx->timing, ctx->rules_version,
                              (ctx->overlap_enabled ? 1 : 0) | (ctx->round_launches ? 2 : 0) |
                                  (ctx->clusters_enabled ? 4 : 0) | (ctx->groups_enabled ? 8 : 0));
  for (auto& g : ctx->graphs) {
    if (g.key == key) {
      g.last_use = ++ctx->graph_clock;
      EEID_CK(cudaGraphLaunch(g.exec, s), "cudaGraphLaunch");
      ctx->launches += g.nkernels;
      return EEID_OK;
    }
  }
  if (!ctx->cap_stream)
    EEID_CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking), "capture stream");
  if (ctx->graphs.size() >= kMaxGraphs) {
    size_t victim = 0;
    for (size_t i = 1; i < ctx->graphs.size(); ++i)
      if (ctx->graphs[i].last_use < ctx->graphs[victim].last_use) victim = i;
    EEID_CK(cudaStreamSynchronize(s), "sync before graph eviction");
    cudaGraphExecDestroy(ctx->graphs[victim].exec);
    cudaFreeHost(ctx->graphs[victim].pinned);
    ctx->graphs.erase(ctx->graphs.begin() + victim);
  }
  eeid_ctx::GraphEntry ge;
  ge.key = std::move(key);
  st = run(ctx, probs, MODE_COMPONENTS, s, &ge);
  if (st != EEID_OK || !ge.exec) {
    if (ge.exec) cudaGraphExecDestroy(ge.exec);
    if (ge.pinned) cudaFreeHost(ge.pinned);
    return st;
  }
  ge.last_use = ++ctx->graph_clock;
  cudaError_t e = cudaGraphLaunch(ge.exec, s);
  if (e != cudaSuccess) {
    cudaGraphExecDestroy(ge.exec);
    cudaFreeHost(ge.pinned);
    return cuda_fail(e, "cudaGraphLaunch");
  }
  ctx->launches += ge.nkernels;
  ctx->graphs.push_back(std::move(ge));
  return EEID_OK;
}

eeid_status eeid_components_host(eeid_ctx* ctx, const double* hA, int64_t lda, int64_t n,
                                 const int64_t* h_rows, int64_t nrows, const int64_t* h_cols,
                                 int64_t ncols, double* h_out, double* h_lambda_opt,
                                 void* stream) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  if (n < 0 || n > kTridiagMaxM) return fail(EEID_ERR_INVALID, "bad n");
  if (n > 0 && (!hA || lda < n)) return fail(EEID_ERR_INVALID, "bad host matrix");
  if (n > 0 && nrows > 0 && ncols > 0 && !h_out) return fail(EEID_ERR_INVALID, "h_out is NULL");
  const int64_t nr = h_rows ? nrows : n, nc = h_cols ? ncols : n;
  if (n == 0 || nr == 0 || nc == 0) return EEID_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // Device copies of A, the grid and the eigenvalues live in a context-owned buffer kept
  // between calls (the context workspace is re-planned by run()); it grows only when a
  // call needs more, so repeated calls of one size allocate nothing.
  const size_t a_bytes = sizeof(double) * (size_t)n * lda;
  const size_t o_bytes = sizeof(double) * (size_t)nr * nc;
  const size_t l_bytes = sizeof(double) * (size_t)n;
  const size_t need = align_up(a_bytes) + align_up(o_bytes) + align_up(l_bytes);
  EEID_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  if (need > ctx->host_call_cap) {
    if (ctx->host_call_buf) {
      cudaError_t e0 = cudaFree(ctx->host_call_buf);   // synchronises the device
      ctx->host_call_buf = nullptr;
      ctx->host_call_cap = 0;
      if (e0 != cudaSuccess) return cuda_fail(e0, "cudaFree(host-call buffer)");
    }
    cudaError_t e0 = cudaMalloc((void**)&ctx->host_call_buf, need);
    if (e0 != cudaSuccess) {
      cudaGetLastError();
      return fail(EEID_ERR_NOMEM, "cudaMalloc(%zu) for the host-call buffer failed", need);
    }
    ctx->host_call_cap = need;
  }
  char* buf = ctx->host_call_buf;
  double* dA = (double*)buf;
  double* dO = (double*)(buf + align_up(a_bytes));
  double* dL = (double*)(buf + align_up(a_bytes) + align_up(o_bytes));
  cudaError_t e = cudaMemcpyAsync(dA, hA, a_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    st = eeid_components(ctx, dA, lda, n, h_rows, nrows, h_cols, ncols, dO,
                         h_lambda_opt ? dL : nullptr, stream);
    if (st == EEID_OK) {
      e = cudaMemcpyAsync(h_out, dO, o_bytes, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess && h_lambda_opt)
        e = cudaMemcpyAsync(h_lambda_opt, dL, l_bytes, cudaMemcpyDeviceToHost, s);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "host-buffer copy");
  if (st != EEID_OK) {
    cudaStreamSynchronize(s);
    return st;
  }
  return eeid_sync(ctx, stream);
}


eeid_status eeid_eigenvectors(eeid_ctx* ctx, const double* dA, int64_t lda, int64_t n,
                              const int64_t* h_rows, int64_t nrows, double* d_vec,
                              double* d_lambda_opt, void* stream) {
  eeid_status st = check_ctx(ctx);
  if (st == EEID_OK) st = check_matrix(dA, lda, n);
  if (st != EEID_OK) return st;
  std::vector<int> rows;
  st = parse_indices(h_rows, nrows, n, "rows", rows);
  if (st != EEID_OK) return st;
  if (n == 0 || nrows == 0) return EEID_OK;
  if (!d_vec) return fail(EEID_ERR_INVALID, "d_vec is NULL");
  EEID_CK(cudaSetDevice(ctx->device), "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const int N = (int)n, NR = (int)nrows;
  // ---- buffers: |v|^2 rows, rotated components, eigenvalues, references, row table
  Arena ar;
  const size_t g_off = ar.take(sizeof(double) * (size_t)NR * N);
  const size_t q_off = ar.take(sizeof(double) * (size_t)NR * std::max(N - 1, 1));
  const size_t l_off = ar.take(sizeof(double) * N);
  const size_t r_off = ar.take(sizeof(int) * (1 + 2 * (size_t)NR));
  const size_t s_off = ar.take(signed_row_bytes() * NR);
  const size_t n_off = ar.take((size_t)NR * N);                 // need[R][N] (R <= NR)
  const size_t p_off = ar.take(sizeof(int) * (size_t)NR * N);   // colpos[R][N]
  if (ar.off > ctx->budget)
    return fail(EEID_ERR_NOMEM, "eigenvector buffers of %zu bytes exceed the HBM budget", ar.off);
  if (ar.off > ctx->vbuf_cap) {
    if (ctx->vbuf) {
      cudaError_t e = cudaFree(ctx->vbuf);   // synchronises the device
      ctx->vbuf = nullptr;
      ctx->vbuf_cap = 0;
      if (e != cudaSuccess) return cuda_fail(e, "cudaFree(eigenvector buffers)");
    }
    cudaError_t e = cudaMalloc((void**)&ctx->vbuf, ar.off);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(EEID_ERR_NOMEM, "cudaMalloc(%zu) for the eigenvector buffers failed", ar.off);
    }
    ctx->vbuf_cap = ar.off;
  }
  const size_t h_bytes = std::max({sizeof(int) * (1 + 2 * (size_t)NR), (size_t)NR * N,
                                   signed_row_bytes() * NR + sizeof(int) * (size_t)NR * N});
  if (ctx->vec_used) EEID_CK(cudaEventSynchronize(ctx->vec_ev), "cudaEventSynchronize(vectors)");
  if (!ctx->vec_ev) EEID_CK(cudaEventCreateWithFlags(&ctx->vec_ev, cudaEventDisableTiming), "event");
  if (h_bytes > ctx->h_vec_cap) {
    if (ctx->h_vec) cudaFreeHost(ctx->h_vec);
    ctx->h_vec = nullptr;
    ctx->h_vec_cap = 0;
    EEID_CK(cudaMallocHost((void**)&ctx->h_vec, h_bytes), "cudaMallocHost(vectors)");
    ctx->h_vec_cap = h_bytes;
  }
  char* vb = ctx->vbuf;
  double* G = (double*)(vb + g_off);
  double* Qg = (double*)(vb + q_off);
  double* lam = d_lambda_opt ? d_lambda_opt : (double*)(vb + l_off);
  int* ri = (int*)(vb + r_off);   // [nref | refs[NR] | row_ref[NR]]
  unsigned char* need = (unsigned char*)(vb + n_off);
  int* colpos = (int*)(vb + p_off);

  // ---- phase 1: |v_ij|^2 for the requested rows, all components j (Eq. 1)
  std::vector<Problem> p1(1);
  p1[0].dA = dA; p1[0].lda = lda; p1[0].n = N; p1[0].rows = rows;
  p1[0].cols.resize(N);
  for (int j = 0; j < N; ++j) p1[0].cols[j] = j;
  p1[0].all_rows = (h_rows == nullptr);
  p1[0].all_cols = true;
  p1[0].out = G;
  p1[0].lam_user = lam;
  st = run(ctx, p1, MODE_COMPONENTS, s);
  if (st != EEID_OK) return st;
  // ---- phase 2: references (greedy cover on the device), read back to plan phase 3
  EEID_CK(launch_pick_refs(G, NR, N, ri + 1, ri + 1 + NR, ri, need, s), "pick_refs launch");
  ctx->launches++;
  int* h_ri = (int*)ctx->h_vec;
  EEID_CK(cudaMemcpyAsync(h_ri, ri, sizeof(int) * (1 + 2 * (size_t)NR), cudaMemcpyDeviceToHost, s),
          "cudaMemcpyAsync(references)");
  EEID_CK(cudaStreamSynchronize(s), "cudaStreamSynchronize(references)");
  const int R = h_ri[0];
  if (R < 0 || R > NR) return fail(EEID_ERR_CUDA, "reference selection returned %d", R);
  std::vector<int> refs(h_ri + 1, h_ri + 1 + R), row_ref(h_ri + 1 + NR, h_ri + 1 + 2 * NR);
  ctx->vec_refs = R;
  // the columns each reference's rows need (|v_ij|^2 not exactly 0 for one of them)
  std::vector<unsigned char> h_need((size_t)R * N);
  if (R > 0) {
    EEID_CK(cudaMemcpyAsync(ctx->h_vec, need, (size_t)R * N, cudaMemcpyDeviceToHost, s),
            "cudaMemcpyAsync(columns needed)");
    EEID_CK(cudaStreamSynchronize(s), "cudaStreamSynchronize(columns needed)");
    memcpy(h_need.data(), ctx->h_vec, (size_t)R * N);
  }
  // ---- phase 3: one problem per reference r: the rotated minors (r, j) for the columns
  // j != r its rows need, for the rows that chose r
  std::vector<Problem> p3;
  std::vector<size_t> q_base(R, 0), q_ncols(R, 0);
  std::vector<int> pos(NR, -1);
  std::vector<int> h_colpos((size_t)R * N, -1);
  size_t qoff = 0;
  for (int q = 0; q < R; ++q) {
    Problem P;
    for (int r = 0; r < NR; ++r)
      if (row_ref[r] == q) { pos[r] = (int)P.rows.size(); P.rows.push_back(rows[r]); }
    for (int j = 0; j < N; ++j)
      if (j != refs[q] && h_need[(size_t)q * N + j]) {
        h_colpos[(size_t)q * N + j] = (int)P.cols.size();
        P.cols.push_back(j);
      }
    q_base[q] = qoff;
    q_ncols[q] = P.cols.size();
    qoff += P.rows.size() * P.cols.size();
    if (P.cols.empty()) continue;   // every other component of these rows is exactly 0
    P.dA = dA; P.lda = lda; P.n = N; P.rot = refs[q]; P.lam_in = lam;
    P.out = Qg + q_base[q];
    p3.push_back(std::move(P));
  }
  if (N >= 2 && !p3.empty()) {
    st = run(ctx, p3, MODE_COMPONENTS, s);
    if (st != EEID_OK) return st;
  }
  // ---- phase 4: assemble the signed vectors and apply the sign convention
  char* h_rows_img = ctx->h_vec;
  int* h_pos_img = (int*)(ctx->h_vec + signed_row_bytes() * NR);
  for (int r = 0; r < NR; ++r) {
    const int q = row_ref[r];
    const double* qrow = q >= 0 ? Qg + q_base[q] + (size_t)pos[r] * q_ncols[q] : nullptr;
    fill_signed_row(h_rows_img + signed_row_bytes() * r, G + (size_t)r * N, qrow,
                    q >= 0 ? colpos + (size_t)q * N : nullptr, d_vec + (size_t)r * N,
                    q >= 0 ? refs[q] : -1);
  }
  if (R > 0) memcpy(h_pos_img, h_colpos.data(), sizeof(int) * (size_t)R * N);
  EEID_CK(cudaMemcpyAsync(vb + s_off, h_rows_img, signed_row_bytes() * NR, cudaMemcpyHostToDevice, s),
          "cudaMemcpyAsync(signed rows)");
  if (R > 0)
    EEID_CK(cudaMemcpyAsync(colpos, h_pos_img, sizeof(int) * (size_t)R * N, cudaMemcpyHostToDevice,
                            s), "cudaMemcpyAsync(column positions)");
  EEID_CK(cudaEventRecord(ctx->vec_ev, s), "cudaEventRecord(vectors)");
  ctx->vec_used = true;
  EEID_CK(launch_signed(vb + s_off, NR, N, s), "signed launch");
  ctx->launches++;
  return EEID_OK;
}


eeid_status eeid_components_herm(eeid_ctx* ctx, const double* dA, int64_t lda, int64_t n,
                                 const int64_t* h_rows, int64_t nrows, const int64_t* h_cols,
                                 int64_t ncols, double* d_out, double* d_lambda_opt,
                                 void* stream) {
  eeid_status st = check_ctx(ctx);
  if (st != EEID_OK) return st;
  if (n > kHermMaxM)
    return fail(EEID_ERR_INVALID, "n = %lld exceeds the Hermitian limit %d", (long long)n, kHermMaxM);
  std::vector<Problem> probs(1);
  st = make_component_problem(dA, lda, n, h_rows, nrows, h_cols, ncols, d_out, d_lambda_opt,
                              probs[0]);
  if (st != EEID_OK) return st;
  probs[0].herm = true;
  if (probs[0].n == 0) return EEID_OK;
  return run(ctx, probs, MODE_COMPONENTS, (cudaStream_t)stream);
}

}  // extern "C"

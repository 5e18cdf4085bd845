// Many reconstructions per launch, and the FFT cluster-size autotuner.
//
// The ptychopy paper runs many small scans by queueing one job per GPU
// (Sec. 3.3, batch GPU mode).  On one B300 a single small scan (J ~ 100..4000
// positions) fills only part of the machine and each of its iterations costs
// a dozen kernel launches.  A batch groups N reconstructions of unequal probe
// size and position count: one iteration of every member is captured once
// into a CUDA graph -- each member's kernels on its own branch, forked from
// and joined back to the batch stream -- and that graph is replayed once per
// iteration, so the members run concurrently and the host issues one launch
// per iteration instead of N x (launches per iteration).
//
// Running every member at once makes their working sets (residuals,
// amplitudes, objects) compete for the 126 MB L2 -- the residuals of a scan
// are re-read four times per iteration -- and was measured slower than
// running them one after another.  So the graph runs the members in groups,
// one group after another: a member whose per-iteration working set reaches
// the group budget forms a group of its own (it fills the GPU by itself), the
// others are packed greedily, largest first, into groups whose working sets
// sum to at most the budget and run concurrently (small scans alone leave
// most SMs idle).  A budget <= 0 puts every member in one group.  The default
// budget, 512 MiB, was the fastest of 0 .. 4 GiB on the 64-scan mixed
// workload of the benchmark.
//
// This file is included by ptycho_api.cu (it uses the context internals).

struct ptycho_batch {
  std::vector<ptycho_ctx*> m;
  std::vector<cudaStream_t> streams;  // one per member, created here
  cudaStream_t main = nullptr;
  bool own_main = false;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  std::vector<cudaEvent_t> gfork;     // one fork event per group
  long long group_bytes = 512LL << 20;
  int lanes = 0;                      // > 0: lanes mode (see batch_plan)
  std::vector<std::vector<int>> groups;  // groups, or in lanes mode the members of each lane in order
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_alg = -1;
  std::vector<char> graph_upd;        // probe-update flag of each member baked into the graph
  long long kernels_per_launch = 0;
  long long graph_launches = 0;
  std::string err;
};

namespace {

thread_local std::string g_batch_error;

int bfail(ptycho_batch* b, int code, const char* fmt, ...) {
  char t[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t, sizeof t, fmt, ap);
  va_end(ap);
  if (b) b->err = t;
  else g_batch_error = t;
  return code;
}

void batch_drop_graph(ptycho_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_alg = -1;
}

// Bytes one iteration of a member streams: the exit-wave / residual array,
// the stored amplitudes and the object-sized arrays.
long long member_bytes(const ptycho_ctx* c) {
  const long long MM = (long long)c->p.M * c->p.M;
  return (long long)c->p.J * MM * (8LL * c->p.K + (c->p.istore == 0 ? 4 : 2)) +
         (long long)c->p.obj_ny * c->p.obj_nx * 24;
}

// Work of one iteration of a member, for the lane assignment: the Fourier
// pass grows as M^2 log2 M per frame, the overlap passes as M^2.
double member_work(const ptycho_ctx* c) {
  const double MM = (double)c->p.M * c->p.M;
  return (double)c->p.J * c->p.K * MM * (std::log2((double)c->p.M) + 6.0);
}

// Partition the members into groups (see the top of this file), or, in lanes
// mode, into `lanes` chains: members sorted by work, largest first, each to
// the chain with the least work so far (longest-processing-time order).  A
// chain runs its members one after another and the chains run side by side,
// so a member starts as soon as its chain's previous member ends, with no
// barrier across chains until the iteration's end.
void batch_plan(ptycho_batch* b) {
  const int n = (int)b->m.size();
  b->groups.clear();
  if (b->lanes > 0) {
    const int L = std::min(b->lanes, n);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return member_work(b->m[x]) > member_work(b->m[y]); });
    b->groups.assign(L, {});
    std::vector<double> load(L, 0.0);
    for (int i : order) {
      const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());  // first least-loaded
      b->groups[l].push_back(i);
      load[l] += member_work(b->m[i]);
    }
  } else if (b->group_bytes <= 0) {
    b->groups.emplace_back();
    for (int i = 0; i < n; ++i) b->groups.back().push_back(i);
  } else {
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return member_bytes(b->m[x]) > member_bytes(b->m[y]); });
    long long cur = 0;
    for (int i : order) {
      const long long w = member_bytes(b->m[i]);
      if (b->groups.empty() || w >= b->group_bytes || cur + w > b->group_bytes) {
        b->groups.emplace_back();
        cur = 0;
      }
      b->groups.back().push_back(i);
      cur += w;
    }
  }
  while (b->gfork.size() < b->groups.size()) {
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    b->gfork.push_back(ev);
  }
}

// Capture one iteration of every member (probe-update flags `upd`) into a
// graph: group after group, the members of a group on parallel branches.
int batch_capture(ptycho_batch* b, int alg, const std::vector<char>& upd) {
  batch_drop_graph(b);
  batch_plan(b);
  cudaError_t e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfail(b, PTYCHO_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
  long long before = 0, after = 0;
  int rc = 0;
  if (b->lanes > 0) {
    // lanes: each member after its chain's previous one, chains side by side
    cudaEventRecord(b->gfork[0], b->main);
    for (size_t l = 0; l < b->groups.size() && !rc; ++l) {
      cudaEvent_t prev = b->gfork[0];
      for (int i : b->groups[l]) {
        ptycho_ctx* c = b->m[i];
        cudaStreamWaitEvent(c->st, prev, 0);
        before += c->launches;
        rc = alg == PTYCHO_DM ? dm_step(c, upd[i] != 0) : lsqml_step(c, upd[i] != 0);
        after += c->launches;
        if (rc) b->err = "member " + std::to_string(i) + ": " + c->err;
        cudaEventRecord(b->join[i], c->st);
        prev = b->join[i];
        if (rc) break;
      }
      cudaStreamWaitEvent(b->main, prev, 0);  // joined even on failure: the capture ends cleanly
    }
  }
  for (size_t g = 0; g < b->groups.size() && !rc && b->lanes <= 0; ++g) {
    cudaEventRecord(b->gfork[g], b->main);  // after the previous group's joins
    for (int i : b->groups[g]) {
      ptycho_ctx* c = b->m[i];
      cudaStreamWaitEvent(c->st, b->gfork[g], 0);
      before += c->launches;
      rc = alg == PTYCHO_DM ? dm_step(c, upd[i] != 0) : lsqml_step(c, upd[i] != 0);
      after += c->launches;
      if (rc) b->err = "member " + std::to_string(i) + ": " + c->err;
      // joined even on failure, so that the capture ends cleanly
      cudaEventRecord(b->join[i], c->st);
      cudaStreamWaitEvent(b->main, b->join[i], 0);
      if (rc) break;
    }
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(b->main, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bfail(b, PTYCHO_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return bfail(b, PTYCHO_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  b->graph = g;
  b->graph_alg = alg;
  b->graph_upd = upd;
  b->kernels_per_launch = after - before;
  return 0;
}

std::mutex g_tune_mu;
std::map<std::pair<int, int>, std::pair<int, double>> g_tune_cache;
std::map<std::pair<int, int>, std::pair<int, double>> g_engine_cache;  // (engine, ms per position)

// k_fill_amp: a deterministic pseudo-random amplitude pattern (tuning data)
__global__ void k_fill_amp(float* a, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)(i * 2654435761u) ^ 0x9e3779b9u;
    h ^= h >> 16;
    a[i] = (float)(h & 0xffff) * (1.0f / 65536.0f);
  }
}

}  // namespace

extern "C" {

int ptycho_autotune(int M, int K, int* best_cluster, double* ms_per_position) {
  if (M < 2 || K < 1) return fail(nullptr, PTYCHO_ERR_ARG, "bad sizes M=%d K=%d", M, K);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find({M, K});
    if (it != g_tune_cache.end()) {
      if (best_cluster) *best_cluster = it->second.first;
      if (ms_per_position) *ms_per_position = it->second.second;
      return PTYCHO_OK;
    }
  }
  // enough positions to fill the GPU several times over (capped at ~512 MB)
  long long J = (512LL << 20) / ((long long)K * M * M * 12);
  if (J > 4096) J = 4096;
  if (J < 64) J = 64;
  const int ny = M + 64, nx = M + 64;
  std::vector<float> pos(2 * J);
  for (long long j = 0; j < J; ++j) {
    pos[2 * j] = (float)((j * 37) % 65);
    pos[2 * j + 1] = (float)((j * 53) % 65);
  }
  int best = 0;
  double best_ms = 1e30;
  for (int C = 1; C <= 16; C *= 2) {
    if (!find_set(M, K, C)) continue;
    ptycho_params p;
    ptycho_default_params(&p);
    p.M = M;
    p.K = K;
    p.J = (int)J;
    p.obj_ny = ny;
    p.obj_nx = nx;
    p.cluster = C;
    ptycho_ctx* ctx = nullptr;
    if (ptycho_create(&ctx, &p) != PTYCHO_OK) continue;  // e.g. shared memory too small
    int rc = set_positions_impl(ctx, pos.data());
    if (!rc) {
      k_fill_amp<<<1184, 256, 0, ctx->st>>>((float*)ctx->amp, (size_t)J * M * M);
      ctx->have_data = true;
      rc = ensure_work_buffers(ctx);
    }
    double ms_min = 1e30;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int rep = 0; rep < 4 && !rc; ++rep) {
      cudaEventRecord(e0, ctx->st);
      rc = launch_fourier(ctx, FM_CHI, ctx->X, nullptr, 0, (int)J, "fourier_chi");
      cudaEventRecord(e1, ctx->st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = PTYCHO_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < ms_min) ms_min = ms;  // first launch is the warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ptycho_destroy(ctx);
    if (!rc && ms_min < best_ms) {
      best_ms = ms_min;
      best = C;
    }
  }
  if (!best) return fail(nullptr, PTYCHO_ERR_UNSUPPORTED, "no runnable kernel for M=%d K=%d", M, K);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[{M, K}] = {best, best_ms / (double)J};
  }
  if (best_cluster) *best_cluster = best;
  if (ms_per_position) *ms_per_position = best_ms / (double)J;
  return PTYCHO_OK;
}

int ptycho_autotune_engine(int M, int K, int* best_engine, int* best_cluster, double* ms_per_position) {
  if (M < 2 || K < 1) return fail(nullptr, PTYCHO_ERR_ARG, "bad sizes M=%d K=%d", M, K);
  int C = 0;
  double ms_reg = 0.0;
  if (int r = ptycho_autotune(M, K, &C, &ms_reg)) return r;
  int eng = PTYCHO_FFT_REGISTER;
  double ms = ms_reg;
  if (M == 64 && K == 1) {
    bool cached = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_engine_cache.find({M, K});
      if (it != g_engine_cache.end()) {
        eng = it->second.first;
        ms = it->second.second;
        cached = true;
      }
    }
    if (!cached) {
      // the tensor-core DFT on the same synthetic residual pass
      const long long J = 4096;
      std::vector<float> pos(2 * J);
      for (long long j = 0; j < J; ++j) {
        pos[2 * j] = (float)((j * 37) % 65);
        pos[2 * j + 1] = (float)((j * 53) % 65);
      }
      ptycho_params p;
      ptycho_default_params(&p);
      p.M = M;
      p.K = K;
      p.J = (int)J;
      p.obj_ny = M + 64;
      p.obj_nx = M + 64;
      p.cluster = C;
      p.fft_engine = PTYCHO_DFT_TENSOR_BF16X3;
      ptycho_ctx* ctx = nullptr;
      double ms_tc = 1e30;
      if (ptycho_create(&ctx, &p) == PTYCHO_OK) {
        int rc = set_positions_impl(ctx, pos.data());
        if (!rc) {
          k_fill_amp<<<1184, 256, 0, ctx->st>>>((float*)ctx->amp, (size_t)J * M * M);
          ctx->have_data = true;
          rc = ensure_work_buffers(ctx);
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int rep = 0; rep < 4 && !rc; ++rep) {
          cudaEventRecord(e0, ctx->st);
          rc = launch_fourier(ctx, FM_CHI, ctx->X, nullptr, 0, (int)J, "fourier_chi");
          cudaEventRecord(e1, ctx->st);
          if (cudaEventSynchronize(e1) != cudaSuccess) rc = PTYCHO_ERR_CUDA;
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          if (rep > 0 && t / (double)J < ms_tc) ms_tc = t / (double)J;  // first launch is the warm-up
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ptycho_destroy(ctx);
        if (rc) ms_tc = 1e30;
      }
      if (ms_tc < ms_reg) {
        eng = PTYCHO_DFT_TENSOR_BF16X3;
        ms = ms_tc;
      }
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_engine_cache[{M, K}] = {eng, ms};
    }
  }
  if (best_engine) *best_engine = eng;
  if (best_cluster) *best_cluster = C;
  if (ms_per_position) *ms_per_position = ms;
  return PTYCHO_OK;
}

int ptycho_batch_create(ptycho_batch** out, int n, const ptycho_params* params, void* stream) {
  if (!out || !params || n < 1) return bfail(nullptr, PTYCHO_ERR_ARG, "bad batch arguments");
  *out = nullptr;
  ptycho_batch* b = new ptycho_batch();
  b->main = (cudaStream_t)stream;
  if (!b->main) {
    cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking);
    b->own_main = true;
  }
  cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < n; ++i) {
    ptycho_params p = params[i];
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      ptycho_batch_destroy(b);
      return bfail(nullptr, PTYCHO_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    }
    b->streams.push_back(s);
    p.stream = s;
    ptycho_ctx* c = nullptr;
    const int rc = ptycho_create(&c, &p);
    if (rc) {
      std::string msg = g_create_error;
      ptycho_batch_destroy(b);
      return bfail(nullptr, rc, "member %d: %s", i, msg.c_str());
    }
    b->m.push_back(c);
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    b->join.push_back(ev);
  }
  *out = b;
  return PTYCHO_OK;
}

ptycho_ctx* ptycho_batch_member(ptycho_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->m.size()) return nullptr;
  return b->m[i];
}

int ptycho_batch_size(const ptycho_batch* b) { return b ? (int)b->m.size() : 0; }

int ptycho_batch_iterate(ptycho_batch* b, int alg, int n_iter) {
  if (!b) return PTYCHO_ERR_ARG;
  if (alg != PTYCHO_DM && alg != PTYCHO_LSQML)
    return bfail(b, PTYCHO_ERR_UNSUPPORTED, "batches run DM or LSQML (ePIE is sequential per scan)");
  if (n_iter < 0) return bfail(b, PTYCHO_ERR_ARG, "n_iter=%d", n_iter);
  for (size_t i = 0; i < b->m.size(); ++i) {
    ptycho_ctx* c = b->m[i];
    if (!c->have_data) return bfail(b, PTYCHO_ERR_STATE, "member %zu has no data", i);
    const int rc = alg == PTYCHO_DM ? dm_prepare(c) : lsqml_prepare(c);
    if (rc) return bfail(b, rc, "member %zu: %s", i, c->err.c_str());
  }
  // the members' own streams must have finished their eager work (uploads,
  // DM initial exit waves) before the graph runs on the batch stream
  for (size_t i = 0; i < b->m.size(); ++i) {
    cudaEventRecord(b->join[i], b->m[i]->st);
    cudaStreamWaitEvent(b->main, b->join[i], 0);
  }
  for (int it = 0; it < n_iter; ++it) {
    std::vector<char> upd(b->m.size());
    for (size_t i = 0; i < b->m.size(); ++i) upd[i] = b->m[i]->t >= b->m[i]->p.probe_start;
    if (!b->exec || b->graph_alg != alg || b->graph_upd != upd)
      if (int rc = batch_capture(b, alg, upd)) return rc;
    cudaError_t e = cudaGraphLaunch(b->exec, b->main);
    if (e != cudaSuccess) return bfail(b, PTYCHO_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    b->graph_launches++;
    for (ptycho_ctx* c : b->m) {
      c->t++;
      if (alg == PTYCHO_DM) c->psi_valid = true;
    }
  }
  // later per-member calls (get_*, fourier_error) on the members' streams
  // must see the graph's results
  cudaEventRecord(b->fork, b->main);
  for (ptycho_ctx* c : b->m) cudaStreamWaitEvent(c->st, b->fork, 0);
  return PTYCHO_OK;
}

long long ptycho_batch_kernels_per_iteration(const ptycho_batch* b) { return b ? b->kernels_per_launch : -1; }

int ptycho_batch_set_group_bytes(ptycho_batch* b, long long bytes) {
  if (!b) return PTYCHO_ERR_ARG;
  if (bytes != b->group_bytes || b->lanes != 0) {
    b->group_bytes = bytes;
    b->lanes = 0;         // groups mode
    batch_drop_graph(b);  // captured again at the next iterate
  }
  return PTYCHO_OK;
}

int ptycho_batch_set_lanes(ptycho_batch* b, int lanes) {
  if (!b) return PTYCHO_ERR_ARG;
  if (lanes < 0) return bfail(b, PTYCHO_ERR_ARG, "lanes=%d", lanes);
  if (lanes != b->lanes) {
    b->lanes = lanes;
    batch_drop_graph(b);
  }
  return PTYCHO_OK;
}

int ptycho_batch_lanes(const ptycho_batch* b) { return b ? b->lanes : -1; }

int ptycho_batch_autotune(ptycho_batch* b, int alg, int n_iter, long long* best_bytes, int* best_lanes,
                          double* best_ms) {
  if (!b) return PTYCHO_ERR_ARG;
  if (n_iter < 1) return bfail(b, PTYCHO_ERR_ARG, "n_iter=%d", n_iter);
  // candidates: group budgets (every member at once, then 64 MiB .. 4 GiB),
  // then lanes of 2 .. 32 chains
  struct Cand {
    long long bytes;
    int lanes;
  };
  std::vector<Cand> cand;
  for (long long gb : {0LL, 64LL << 20, 128LL << 20, 256LL << 20, 512LL << 20, 1LL << 30, 2LL << 30, 4LL << 30})
    cand.push_back({gb, 0});
  for (int l : {2, 4, 8, 16, 32})
    if (l < (int)b->m.size()) cand.push_back({b->group_bytes, l});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return bfail(b, PTYCHO_ERR_CUDA, "event creation failed");
  Cand best{b->group_bytes, b->lanes};
  float best_t = -1.f;
  int rc = PTYCHO_OK;
  std::vector<std::pair<int, std::vector<std::vector<int>>>> seen;  // schedules already timed
  for (const Cand& cd : cand) {
    if (cd.lanes > 0) {
      if ((rc = ptycho_batch_set_lanes(b, cd.lanes))) break;
    } else if ((rc = ptycho_batch_set_group_bytes(b, cd.bytes))) {
      break;
    }
    batch_plan(b);
    const std::pair<int, std::vector<std::vector<int>>> key{cd.lanes > 0, b->groups};
    if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;  // same schedule as before
    seen.push_back(key);
    if ((rc = ptycho_batch_iterate(b, alg, 1))) break;  // captures the graph of this schedule
    cudaEventRecord(e0, b->main);
    if ((rc = ptycho_batch_iterate(b, alg, n_iter))) break;
    cudaEventRecord(e1, b->main);
    float t = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      rc = bfail(b, PTYCHO_ERR_CUDA, "timing failed");
      break;
    }
    if (best_t < 0.f || t < best_t) {
      best_t = t;
      best = cd;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (int r = ptycho_batch_set_group_bytes(b, best.bytes)) return r;
  if (best.lanes > 0)
    if (int r = ptycho_batch_set_lanes(b, best.lanes)) return r;
  if (best_bytes) *best_bytes = best.bytes;
  if (best_lanes) *best_lanes = best.lanes;
  if (best_ms) *best_ms = best_t / n_iter;
  return PTYCHO_OK;
}

int ptycho_batch_groups(ptycho_batch* b, int* group_of) {
  if (!b) return -1;
  batch_plan(b);
  if (group_of)
    for (size_t g = 0; g < b->groups.size(); ++g)
      for (int i : b->groups[g]) group_of[i] = (int)g;
  return (int)b->groups.size();
}

int ptycho_batch_synchronize(ptycho_batch* b) {
  if (!b) return PTYCHO_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(b->main);
  if (e != cudaSuccess) return bfail(b, PTYCHO_ERR_CUDA, "synchronize: %s", cudaGetErrorString(e));
  return PTYCHO_OK;
}

const char* ptycho_batch_last_error(const ptycho_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

void ptycho_batch_destroy(ptycho_batch* b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  batch_drop_graph(b);
  for (ptycho_ctx* c : b->m) ptycho_destroy(c);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  for (cudaEvent_t e : b->gfork) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->own_main) cudaStreamDestroy(b->main);
  delete b;
}

}  // extern "C"

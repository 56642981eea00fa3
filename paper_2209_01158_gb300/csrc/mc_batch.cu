// Batched precision form: many independent instances (each an mc_ctx of its
// own grid size and number of continua) advanced together, one persistent
// launch per time step for the whole batch, the launches of a call captured
// once into a CUDA graph and replayed. Also the team-size autotuner and its
// JSON cache.

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <map>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "mc_internal.h"

struct mc_batch {
  int device = 0;
  cudaStream_t stream = nullptr;       // own non-blocking stream (graph capture)
  std::vector<cudaStream_t> ctx_streams;
  cudaEvent_t ev = nullptr;
  int n = 0;
  int bf16 = 0;
  std::vector<mc_ctx*> ctx;
  std::vector<int> order;              // largest first
  mc_opts opts{};
  int num_sms = 0;
  int max_blocks = 0;                  // co-resident CTAs of the batched kernel
  int team = 0, teams = 0;
  IrParams* d_ip = nullptr;
  TmaMaps* d_maps = nullptr;
  int* d_order = nullptr;
  BatchInst* d_st = nullptr;
  unsigned* d_ctrl = nullptr;
  size_t ctrl_bytes = 0;
  unsigned* d_abort = nullptr;
  double* d_partials = nullptr;
  std::vector<BatchInst> h_st;
  std::vector<BatchInst> h_init;       // records at the start of a call
  // instances whose FP32 refinement failed once: stepped by the FP64 PCG path
  std::vector<char> fp64;
  int n_fp64 = 0;
  // the captured time loop
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string graph_key;
  int graph_used = 0;
  int tuned_from_cache = 0;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  std::string err;
};

namespace {

thread_local std::string g_batch_err;

mc_status berr(mc_batch* b, mc_status s, const std::string& msg) {
  if (b) b->err = msg; else g_batch_err = msg;
  return s;
}

#define BK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return berr(b, MC_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

cudaError_t balloc(mc_batch* b, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 8;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return e;
  b->allocs.push_back(*p);
  b->bytes += (int64_t)bytes;
  return cudaMemset(*p, 0, bytes);
}

void bfree(mc_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->stream) cudaStreamDestroy(b->stream);
}

// Work of one step of an instance, up to a constant: L N cells times a PCG
// iteration count that grows like the grid's side (Jacobi on a 2-D stencil).
double inst_cost(const mc_ctx* c) {
  return (double)c->L * (double)c->N * (double)std::max(c->nx, c->ny);
}

// Default team size: small teams amortise barrier latency over more
// concurrent instances; the team must still be large enough that the largest
// instance does not outlast the rest of the batch (cost_max / team <=
// total / blocks). Rounded up to a power of two.
int default_team(const mc_batch* b, int blocks) {
  double tot = 0.0, mx = 0.0;
  for (const mc_ctx* c : b->ctx) {
    const double w = inst_cost(c);
    tot += w;
    mx = std::max(mx, w);
  }
  const double need = tot > 0.0 ? mx * blocks / tot : 1.0;
  int g = 1;
  while (g < need && g < blocks) g *= 2;
  return std::min(g, blocks);
}

int launch_blocks(const mc_batch* b) {
  int blocks = b->max_blocks;
  if (b->opts.blocks > 0 && b->opts.blocks < blocks) blocks = b->opts.blocks;
  return blocks;
}

BatchParams make_params(const mc_batch* b, int scheme) {
  BatchParams bp;
  memset(&bp, 0, sizeof(bp));
  bp.inst = b->d_ip;
  bp.maps = b->d_maps;
  bp.order = b->d_order;
  bp.st = b->d_st;
  bp.n = b->n;
  bp.team = b->team;
  bp.teams = b->teams;
  bp.scheme = scheme;
  bp.rtol = b->opts.rtol;
  bp.inner_rtol = b->opts.inner_rtol;
  bp.max_iter = b->opts.max_iter;
  bp.ir_max = b->opts.ir_max;
  bp.inner_form = b->opts.inner_form;
  bp.spin_limit = b->opts.spin_limit;
  bp.ctrl = b->d_ctrl;
  bp.abort_word = b->d_abort;
  bp.partials = b->d_partials;
  return bp;
}

// Queue one batched step (control words zeroed, then the launch).
cudaError_t queue_step(mc_batch* b, const BatchParams& bp) {
  cudaError_t e = cudaMemsetAsync(b->d_ctrl, 0, b->ctrl_bytes, b->stream);
  if (e != cudaSuccess) return e;
  return mc_launch_ir_batch(bp, b->bf16, b->team * b->teams, b->stream);
}

// The members' streams finish their queued work (state, sources) before the
// batch stream starts.
cudaError_t join_members(mc_batch* b) {
  for (cudaStream_t s : b->ctx_streams) {
    cudaError_t e = cudaEventRecord(b->ev, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(b->stream, b->ev, 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Keep every member's low-precision copies in the batch's format (a member
// stepped alone in the other format in between rewrites them).
cudaError_t refresh_members(mc_batch* b) {
  for (mc_ctx* c : b->ctx) {
    if (c->lo_kind != 1 + b->bf16) {
      cudaError_t e = mc_ir_prepare(c, b->bf16);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// After a timed-out launch: instances a team held mid-step go back to the
// start of that step (p <- p^{n-1}).
cudaError_t restore_busy(mc_batch* b) {
  for (int i = 0; i < b->n; ++i) {
    if (!b->h_st[i].busy) continue;
    mc_ctx* c = b->ctx[i];
    for (int a = 0; a < c->L; ++a) {
      cudaError_t e = cudaMemcpyAsync(c->p[a], c->pprev[a], (size_t)c->Np * sizeof(double),
                                      cudaMemcpyDeviceToDevice, b->stream);
      if (e != cudaSuccess) return e;
    }
    if (b->h_st[i].status == 0) b->h_st[i].status = MC_E_TIMEOUT;
  }
  return cudaSuccess;
}

// Undo the last step of every batched instance (p <- p^{n-1}); used by the
// tuner (instances on the FP64 path are skipped by the trial launches).
cudaError_t undo_step(mc_batch* b) {
  for (int i = 0; i < b->n; ++i) {
    if (b->fp64[i]) continue;
    mc_ctx* c = b->ctx[i];
    for (int a = 0; a < c->L; ++a) {
      cudaError_t e = cudaMemcpyAsync(c->p[a], c->pprev[a], (size_t)c->Np * sizeof(double),
                                      cudaMemcpyDeviceToDevice, b->stream);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// Zeroed records; instances on the FP64 path carry a nonzero status so the
// batched kernel skips them.
constexpr int kSkip = -1;

cudaError_t reset_records(mc_batch* b) {
  b->h_init.assign(b->n, BatchInst{});
  for (int i = 0; i < b->n; ++i)
    if (b->fp64[i]) b->h_init[i].status = kSkip;
  cudaError_t e = cudaMemcpyAsync(b->d_st, b->h_init.data(), sizeof(BatchInst) * b->n,
                                  cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(b->d_abort, 0, 128, b->stream);
}

// nsteps steps of instance i by the FP64 PCG path (mc_step_decoupled with
// the batch's tolerances), added to its record.
mc_status fp64_steps(mc_batch* b, int i, int scheme, int nsteps) {
  mc_ctx* c = b->ctx[i];
  const mc_opts save = c->opts;
  c->opts.precision = MC_PREC_FP64;
  c->opts.precond = b->opts.precond;
  c->opts.rtol = b->opts.rtol;
  c->opts.max_iter = b->opts.max_iter;
  c->opts.spin_limit = b->opts.spin_limit;
  c->opts.blocks = 0;
  mc_stats s;
  const mc_status st = mc_step_decoupled(c, scheme, nsteps, &s);
  c->opts = save;
  BatchInst& r = b->h_st[i];
  r.steps_done += s.steps_done;
  r.status = s.status ? s.status : (st == MC_OK ? 0 : (int)st);
  for (int a = 0; a < MCL; ++a) {
    r.iters[a] += s.iters[a];
    r.max_iters[a] = std::max(r.max_iters[a], s.max_iters[a]);
    r.relres[a] = s.rel_residual[a];
  }
  return st;
}

cudaError_t fetch_records(mc_batch* b, unsigned* abort_word) {
  cudaError_t e = cudaMemcpyAsync(b->h_st.data(), b->d_st, sizeof(BatchInst) * b->n,
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(abort_word, b->d_abort, sizeof(unsigned), cudaMemcpyDeviceToHost,
                           b->stream)) != cudaSuccess)
    return e;
  return cudaStreamSynchronize(b->stream);
}

void fill_stats(const BatchInst& r, mc_stats* s) {
  memset(s, 0, sizeof(*s));
  s->steps_done = r.steps_done;
  s->status = r.status;
  for (int a = 0; a < MCL; ++a) {
    s->iters[a] = r.iters[a];
    s->max_iters[a] = r.max_iters[a];
    s->rel_residual[a] = r.relres[a];
  }
  s->ir_sweeps = r.ir_sweeps;
}

// ---- autotuner cache: a flat JSON object, one entry per line -------------------
//   "key": {"team": 8, "ms": 12.345},
std::string tune_key(const mc_batch* b, int scheme, int blocks) {
  cudaDeviceProp prop;
  std::string dev = "unknown";
  int cc = 0;
  if (cudaGetDeviceProperties(&prop, b->device) == cudaSuccess) {
    dev = prop.name;
    cc = prop.major * 10 + prop.minor;
  }
  for (char& ch : dev)
    if (ch == '"' || ch == '\\' || ch == '|') ch = '_';
  // FNV-1a over the sorted (nx, ny, L) list: the key depends on the batch's
  // composition, not on the order the instances were given in
  std::vector<long long> shapes;
  for (const mc_ctx* c : b->ctx)
    shapes.push_back(((long long)c->nx << 32) ^ ((long long)c->ny << 4) ^ (long long)c->L);
  std::sort(shapes.begin(), shapes.end());
  unsigned long long h = 1469598103934665603ull;
  for (long long v : shapes)
    for (int k = 0; k < 8; ++k) {
      h ^= (unsigned long long)((v >> (8 * k)) & 0xff);
      h *= 1099511628211ull;
    }
  char buf[256];
  snprintf(buf, sizeof(buf), "%s|sm%d|%s|scheme%d|n%d|blocks%d|%016llx", dev.c_str(), cc,
           b->bf16 ? "bf16t" : "fp32", scheme, b->n, blocks, h);
  return buf;
}

std::map<std::string, std::pair<int, double>> read_cache(const char* path) {
  std::map<std::string, std::pair<int, double>> m;
  std::ifstream f(path);
  if (!f) return m;
  std::string line;
  while (std::getline(f, line)) {
    const size_t q0 = line.find('"');
    if (q0 == std::string::npos) continue;
    const size_t q1 = line.find('"', q0 + 1);
    if (q1 == std::string::npos) continue;
    const std::string key = line.substr(q0 + 1, q1 - q0 - 1);
    const size_t t = line.find("\"team\":", q1);
    const size_t ms = line.find("\"ms\":", q1);
    if (t == std::string::npos) continue;
    const int team = atoi(line.c_str() + t + 7);
    const double tms = ms == std::string::npos ? -1.0 : atof(line.c_str() + ms + 5);
    if (team > 0) m[key] = {team, tms};
  }
  return m;
}

bool write_cache(const char* path, const std::map<std::string, std::pair<int, double>>& m) {
  const std::string tmp = std::string(path) + ".tmp";
  {
    std::ofstream f(tmp);
    if (!f) return false;
    f << "{\n";
    size_t k = 0;
    for (const auto& kv : m) {
      char buf[64];
      snprintf(buf, sizeof(buf), "%.6f", kv.second.second);
      f << "  \"" << kv.first << "\": {\"team\": " << kv.second.first << ", \"ms\": " << buf << "}"
        << (++k < m.size() ? ",\n" : "\n");
    }
    f << "}\n";
    if (!f) return false;
  }
  return rename(tmp.c_str(), path) == 0;
}

void set_team(mc_batch* b, int team) {
  const int blocks = launch_blocks(b);
  b->team = std::max(1, std::min(team, blocks));
  b->teams = blocks / b->team;
}

}  // namespace

extern "C" {

const char* mc_batch_last_error(const mc_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

mc_status mc_batch_create(mc_ctx* const* ctxs, int32_t n, const mc_opts* opts, mc_batch** out) {
  mc_batch* b = nullptr;
  if (!out) return berr(nullptr, MC_E_ARG, "out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1) return berr(nullptr, MC_E_ARG, "need n >= 1 contexts");
  if (!opts) return berr(nullptr, MC_E_ARG, "opts is NULL");
  if (opts->precision != MC_PREC_FP32_IR && opts->precision != MC_PREC_BF16T_IR)
    return berr(nullptr, MC_E_ARG, "the batched form needs precision MC_PREC_FP32_IR or MC_PREC_BF16T_IR");
  if (opts->max_iter < 1 || !(opts->rtol > 0.0) || !(opts->rtol < 1.0) || opts->spin_limit < 1 ||
      opts->blocks < 0 || opts->ir_max < 0 || !(opts->inner_rtol > 0.0) || !(opts->inner_rtol < 1.0) ||
      (opts->inner_form != MC_INNER_SINGLE_REDUCTION && opts->inner_form != MC_INNER_TWO_REDUCTIONS) ||
      (opts->precond != MC_PRECOND_JACOBI && opts->precond != MC_PRECOND_TWO_LEVEL))
    return berr(nullptr, MC_E_ARG, "opts out of range");
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return berr(nullptr, MC_E_ARG, "context " + std::to_string(i) + " is NULL");
  for (int i = 1; i < n; ++i)
    if (ctxs[i]->device != ctxs[0]->device)
      return berr(nullptr, MC_E_ARG, "all contexts must live on one device");
  b = new (std::nothrow) mc_batch;
  if (!b) return berr(nullptr, MC_E_ALLOC, "host allocation failed");
  b->device = ctxs[0]->device;
  b->n = n;
  b->opts = *opts;
  b->bf16 = opts->precision == MC_PREC_BF16T_IR ? 1 : 0;
  b->ctx.assign(ctxs, ctxs + n);
  b->h_st.assign(n, BatchInst{});
  b->fp64.assign(n, 0);
  auto fail = [&](mc_status s) {
    g_batch_err = b->err;
    bfree(b);
    delete b;
    return s;
  };
  mc_status st = MC_OK;
  {
    cudaError_t e;
#define BC(call)                                                                   \
  if ((e = (call)) != cudaSuccess) {                                               \
    berr(b, MC_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e));          \
    return fail(MC_E_CUDA);                                                        \
  }
    BC(cudaSetDevice(b->device));
    BC(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    BC(cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming));
    BC(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device));
    for (mc_ctx* c : b->ctx)
      if (std::find(b->ctx_streams.begin(), b->ctx_streams.end(), c->stream) == b->ctx_streams.end())
        b->ctx_streams.push_back(c->stream);
    for (mc_ctx* c : b->ctx) BC(mc_ir_prepare(c, b->bf16));
    for (cudaStream_t s : b->ctx_streams) BC(cudaStreamSynchronize(s));
    b->max_blocks = mc_ir_batch_max_blocks(b->bf16 != 0, b->num_sms);
    if (b->max_blocks < 1) {
      berr(b, MC_E_CUDA, "no co-resident CTAs for the batched kernel");
      return fail(MC_E_CUDA);
    }
    const int blocks = launch_blocks(b);
    std::vector<IrParams> ip(n);
    std::vector<TmaMaps> maps(n);
    for (int i = 0; i < n; ++i) {
      StepParams sp;
      mc_fill_params(b->ctx[i], &sp, MC_SCHEME_D, 1);
      mc_ir_fill(b->ctx[i], sp, &ip[i]);
      maps[i] = b->ctx[i]->maps32;
    }
    b->order.resize(n);
    for (int i = 0; i < n; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
      return inst_cost(b->ctx[x]) > inst_cost(b->ctx[y]);
    });
    BC(balloc(b, (void**)&b->d_ip, sizeof(IrParams) * n));
    BC(balloc(b, (void**)&b->d_maps, sizeof(TmaMaps) * n));
    BC(balloc(b, (void**)&b->d_order, sizeof(int) * n));
    BC(balloc(b, (void**)&b->d_st, sizeof(BatchInst) * n));
    b->ctrl_bytes = sizeof(unsigned) * 32 * (size_t)(blocks + 1);
    BC(balloc(b, (void**)&b->d_ctrl, b->ctrl_bytes));
    BC(balloc(b, (void**)&b->d_abort, 128));
    BC(balloc(b, (void**)&b->d_partials, sizeof(double) * 2 * MC_KMAX_ALLOC * (size_t)blocks));
    BC(cudaMemcpy(b->d_ip, ip.data(), sizeof(IrParams) * n, cudaMemcpyHostToDevice));
    BC(cudaMemcpy(b->d_maps, maps.data(), sizeof(TmaMaps) * n, cudaMemcpyHostToDevice));
    BC(cudaMemcpy(b->d_order, b->order.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
#undef BC
    set_team(b, default_team(b, blocks));
  }
  *out = b;
  return st;
}

mc_status mc_batch_set_team(mc_batch* b, int32_t team) {
  if (!b) return MC_E_ARG;
  if (team < 1 || team > launch_blocks(b))
    return berr(b, MC_E_ARG, "team must be in 1.." + std::to_string(launch_blocks(b)));
  set_team(b, team);
  return MC_OK;
}

mc_status mc_batch_step(mc_batch* b, int32_t scheme, int32_t nsteps, mc_stats* total) {
  if (!b) return MC_E_ARG;
  if (total) memset(total, 0, sizeof(*total));
  if (scheme != MC_SCHEME_D && scheme != MC_SCHEME_L && scheme != MC_SCHEME_U)
    return berr(b, MC_E_ARG, "scheme must be MC_SCHEME_D, _L or _U");
  if (nsteps < 0) return berr(b, MC_E_ARG, "nsteps < 0");
  if (nsteps == 0) return MC_OK;
  BK(cudaSetDevice(b->device));
  BK(refresh_members(b));
  BK(join_members(b));
  BK(reset_records(b));
  const BatchParams bp = make_params(b, scheme);
  const std::string key = std::to_string(scheme) + "/" + std::to_string(nsteps) + "/" +
                          std::to_string(b->team) + "/" + std::to_string(b->teams);
  if (b->exec && b->graph_key != key) {
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
  }
  if (!b->exec) {
    // capture the whole time loop once; replays reuse it
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int s = 0; s < nsteps && e == cudaSuccess; ++s) e = queue_step(b, bp);
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      b->exec = nullptr;
      return berr(b, MC_E_CUDA, std::string("graph capture of the batched time loop: ") +
                                    cudaGetErrorString(e));
    }
    b->graph = g;
    b->graph_key = key;
  }
  BK(cudaGraphLaunch(b->exec, b->stream));
  b->graph_used = 1;
  unsigned abort_word = 0;
  BK(fetch_records(b, &abort_word));
  if (abort_word) {
    BK(restore_busy(b));
    BK(cudaStreamSynchronize(b->stream));
  } else {
    // FP32 refinement that failed (MC_E_NOCONV: the instance is back at the
    // start of its failed step) hands the instance to the FP64 PCG path for
    // the rest of this call and for later calls; instances already there
    // take all their steps by it.
    for (int i = 0; i < b->n; ++i) {
      BatchInst& r = b->h_st[i];
      if (r.status == kSkip) {
        r.status = 0;
      } else if (r.status == MC_E_NOCONV) {
        b->fp64[i] = 1;
        ++b->n_fp64;
        r.status = 0;
      } else {
        continue;
      }
      fp64_steps(b, i, scheme, nsteps - r.steps_done);
    }
  }
  mc_stats acc;
  memset(&acc, 0, sizeof(acc));
  acc.steps_done = nsteps;
  int bad = -1;
  for (int i = 0; i < b->n; ++i) {
    const BatchInst& r = b->h_st[i];
    acc.steps_done = std::min(acc.steps_done, r.steps_done);
    for (int a = 0; a < MCL; ++a) {
      acc.iters[a] += r.iters[a];
      acc.max_iters[a] = std::max(acc.max_iters[a], r.max_iters[a]);
    }
    acc.ir_sweeps += r.ir_sweeps;
    if (r.status != 0 && bad < 0) bad = i;
  }
  if (abort_word && bad < 0) bad = 0;
  acc.status = bad >= 0 ? (b->h_st[bad].status ? b->h_st[bad].status : (int)MC_E_TIMEOUT) : 0;
  if (total) *total = acc;
  if (bad >= 0)
    return berr(b, (mc_status)acc.status,
                "instance " + std::to_string(bad) + " stopped after " +
                    std::to_string(b->h_st[bad].steps_done) + " steps: " +
                    mc_status_string((mc_status)acc.status));
  return MC_OK;
}

mc_status mc_batch_instance_stats(mc_batch* b, int32_t i, mc_stats* s) {
  if (!b || !s || i < 0 || i >= b->n) return MC_E_ARG;
  fill_stats(b->h_st[i], s);
  return MC_OK;
}

mc_status mc_batch_autotune(mc_batch* b, int32_t scheme, const int32_t* candidates, int32_t ncand,
                            const char* cache_path, int32_t* best_team, double* ms) {
  if (!b) return MC_E_ARG;
  if (scheme != MC_SCHEME_D && scheme != MC_SCHEME_L && scheme != MC_SCHEME_U)
    return berr(b, MC_E_ARG, "scheme must be MC_SCHEME_D, _L or _U");
  const int blocks = launch_blocks(b);
  std::vector<int> cand;
  if (candidates && ncand > 0) {
    for (int k = 0; k < ncand; ++k)
      if (candidates[k] >= 1 && candidates[k] <= blocks) cand.push_back(candidates[k]);
  } else {
    for (int g = 1; g <= blocks; g *= 2) cand.push_back(g);
    if (cand.back() != blocks) cand.push_back(blocks);
  }
  if (ms)
    for (int k = 0; k < ncand; ++k) ms[k] = -1.0;
  if (cand.empty()) return berr(b, MC_E_ARG, "no admissible team size among the candidates");
  const std::string key = tune_key(b, scheme, blocks);
  b->tuned_from_cache = 0;
  if (cache_path) {
    auto m = read_cache(cache_path);
    auto it = m.find(key);
    if (it != m.end() && it->second.first >= 1 && it->second.first <= blocks) {
      set_team(b, it->second.first);
      b->tuned_from_cache = 1;
      if (best_team) *best_team = b->team;
      return MC_OK;
    }
  }
  BK(cudaSetDevice(b->device));
  BK(refresh_members(b));
  BK(join_members(b));
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0));
  BK(cudaEventCreate(&e1));
  double best = 1e300;
  int best_g = b->team;
  mc_status st = MC_OK;
  // one untimed step first (first-launch costs), then one timed step per
  // candidate; every trial step is undone, so the state is left unchanged
  for (int k = -1; k < (int)cand.size() && st == MC_OK; ++k) {
    set_team(b, k < 0 ? cand[0] : cand[k]);
    const BatchParams bp = make_params(b, scheme);
    cudaError_t e = reset_records(b);
    if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
    if (e == cudaSuccess) e = queue_step(b, bp);
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
    unsigned abort_word = 0;
    if (e == cudaSuccess) e = fetch_records(b, &abort_word);
    if (e != cudaSuccess) {
      st = berr(b, MC_E_CUDA, std::string("autotune step: ") + cudaGetErrorString(e));
      break;
    }
    if (abort_word) {
      restore_busy(b);
      cudaStreamSynchronize(b->stream);
      st = berr(b, MC_E_TIMEOUT, "autotune step timed out");
      break;
    }
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if ((e = undo_step(b)) != cudaSuccess || (e = cudaStreamSynchronize(b->stream)) != cudaSuccess) {
      st = berr(b, MC_E_CUDA, std::string("autotune undo: ") + cudaGetErrorString(e));
      break;
    }
    if (k < 0) continue;
    if (ms && candidates && ncand > 0) {
      for (int j = 0; j < ncand; ++j)
        if (candidates[j] == cand[k]) ms[j] = t;
    } else if (ms && k < ncand) {
      ms[k] = t;
    }
    if (t < best) {
      best = t;
      best_g = cand[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  reset_records(b);
  cudaStreamSynchronize(b->stream);
  set_team(b, best_g);
  if (st != MC_OK) return st;
  if (best_team) *best_team = b->team;
  if (cache_path) {
    auto m = read_cache(cache_path);
    m[key] = {b->team, best};
    if (!write_cache(cache_path, m)) return berr(b, MC_E_ARG, std::string("cannot write ") + cache_path);
  }
  return MC_OK;
}

mc_status mc_batch_info(const mc_batch* b, int64_t* info) {
  if (!b || !info) return MC_E_ARG;
  double cells = 0.0;
  for (const mc_ctx* c : b->ctx) cells += (double)c->L * (double)c->N;
  info[0] = b->n;
  info[1] = b->team;
  info[2] = b->teams;
  info[3] = b->team * b->teams;
  info[4] = b->graph_used;
  info[5] = b->tuned_from_cache;
  info[6] = (int64_t)cells;
  info[7] = b->bytes;
  info[8] = b->n_fp64;
  return MC_OK;
}

void mc_batch_destroy(mc_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  bfree(b);
  delete b;
}

}  // extern "C"

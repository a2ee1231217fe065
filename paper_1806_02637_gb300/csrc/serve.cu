// Serving: motion-compensation jobs (precompute once, then gradient iterations of
// the consistency) scheduled by continuous batching on one device.
//
// Two host threads per serving context:
//   admission  takes queued jobs in arrival order while the device-memory budget
//              and the slot limit allow, allocates the job's memory (stream-ordered),
//              copies its inputs and runs its dRadon/ds precompute on the admission
//              stream; then frees the precompute's transient memory and hands the job
//              to the round loop.  Precompute of new jobs overlaps the rounds.
//   rounds     while jobs are active, issues one round after another on the round
//              stream: every active job does one evaluation (and, until its last
//              round, one gradient step).  A round is a fixed sequence of launches
//              over a device table of the active jobs: view and pair set-up, one
//              persistent pair launch over all jobs' pair blocks, per-job totals,
//              pair gradients, per-view gradient sums and the steps.  Jobs join at the
//              next round after their precompute and leave after their last one;
//              their results go to pinned host memory and the job's memory is freed.
// Every per-job reduction has a fixed order, so a job's results do not depend on
// which other jobs share its rounds.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ecc.h"
#include "ecc_internal.cuh"
#include "kernels.cuh"
#include "serve.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxActive = 64;              // jobs per round
constexpr size_t kSlotBytes = 256 * 1024;   // pinned result staging per job
constexpr int kMaxViewsServed = 4096;
constexpr int kMaxIters = 100000;
constexpr int kWarpsPerPairBlock = 8;       // pairs per block of the pair kernel

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

size_t elem_size(int dtype) { return dtype == ECC_F32 ? 4 : 2; }

struct Layout {  // byte offsets of a job's resident and transient sections
  size_t P, theta, grad, views, vtan, adir, sino, scales, prs, ctile, partial, Gpp, gpp, totals, status;
  size_t theta0, nodes, jac, jbase, resident;
  size_t images, rtable, wimg, stage, transient;
  int batch;
};

Layout layout_of(const ecc_job& j) {
  Layout L{};
  const size_t n = (size_t)j.n_views;
  const size_t np = n * (n - 1) / 2;
  const size_t n_tiles = ((size_t)j.n_kappa + 31) / 32;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + (bytes ? bytes : 16));
    return at;
  };
  L.P = take(n * 12 * sizeof(double));
  L.theta = take(n * 6 * sizeof(double));
  L.grad = take(n * 6 * sizeof(double));
  L.views = take(n * sizeof(ecc::ViewRec));
  L.vtan = take(n * sizeof(ecc::ViewTan));
  L.adir = take((size_t)j.n_alpha * sizeof(float4));
  L.sino = take(n * (size_t)j.n_alpha * j.n_s * elem_size(j.dtype));
  L.scales = take(n * sizeof(float));
  L.prs = take(np * sizeof(ecc::PairRec));
  L.ctile = take(np * n_tiles * sizeof(float4));
  L.partial = take((np + kWarpsPerPairBlock - 1) / kWarpsPerPairBlock * sizeof(double));
  L.Gpp = take(np * 12 * sizeof(double));
  L.gpp = take(np * 30 * sizeof(float2));
  L.totals = take(((size_t)j.n_iters + 1) * sizeof(double));
  L.status = take(sizeof(int));
  L.theta0 = take(n * 6 * sizeof(double));
  const size_t nn = j.motion_model == ECC_MOTION_AKIMA ? (size_t)j.n_nodes : 0;
  L.nodes = take(nn * 6 * sizeof(double));
  L.jac = take(nn ? n * 36 * sizeof(double) : 0);
  L.jbase = take(nn ? n * 6 * sizeof(int) : 0);
  L.resident = o;
  o = 0;
  L.images = take(n * (size_t)j.W * j.H * sizeof(float));
  L.rtable = take(n * (size_t)j.n_alpha * sizeof(ecc::RadonRow) + n * sizeof(ecc::RadonView));
  const size_t plane = ecc::radon_plane_bytes(j.W, j.H, j.n_s);
  L.batch = (int)std::max<size_t>(1, std::min<size_t>(n, ((size_t)256 << 20) / plane));
  L.wimg = take(plane * (size_t)L.batch);
  L.stage = take(j.dtype == ECC_F16 ? ecc::radon_f16_stage_bytes(j.n_alpha, j.n_s, L.batch) : 0);
  L.transient = o;
  return L;
}

enum class State { Queued, Admitting, Active, Finishing, Done, Failed };

struct Job {
  uint64_t ticket = 0;
  ecc_job d{};
  Layout L{};
  State st = State::Queued;
  unsigned char* dev = nullptr;  // resident block
  unsigned char* tmp = nullptr;  // transient block (precompute)
  double* h_stage = nullptr;     // pinned slot: totals [n_iters + 1], theta [n_views][6]
  int slot = -1;
  int rounds = 0;                // evaluations issued
  cudaEvent_t done = nullptr;
  Clock::time_point t_submit, t_admit, t_done;
  int err = ECC_OK;
  std::string msg;
  ecc_result res{};
};

}  // namespace

struct ecc_serve {
  int device = 0;
  size_t budget = 0;
  size_t used = 0;
  std::mutex mu;
  std::condition_variable cv_admit, cv_round;
  std::thread th_admit, th_round;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<Job*> queue;
  std::vector<Job*> ready;     // admitted, waiting for the next round
  std::unordered_map<uint64_t, Job*> jobs;
  int admitting = 0, running = 0;  // jobs in admission / in rounds or finishing
  cudaStream_t s_admit = nullptr, s_round = nullptr;
  // round table: device copy and a pinned ring of two host copies
  ecc::ServeJob* d_jobs = nullptr;
  long long* d_off = nullptr;
  unsigned long long* d_counter = nullptr;
  ecc::ServeJob* h_jobs[2] = {nullptr, nullptr};
  long long* h_off[2] = {nullptr, nullptr};
  cudaEvent_t round_ev[2] = {nullptr, nullptr};
  // device time: timing events around each round (one pair per ring slot, read once
  // the slot's round has completed) and around each admission's copies and precompute
  cudaEvent_t round_t0[2] = {nullptr, nullptr}, round_t1[2] = {nullptr, nullptr};
  bool round_pending[2] = {false, false};
  cudaEvent_t admit_t[3] = {nullptr, nullptr, nullptr};
  double round_ms = 0.0, upload_ms = 0.0, precompute_ms = 0.0;
  int pair_grid = 0;
  // pinned result slots
  unsigned char* slots = nullptr;
  std::vector<int> free_slots;
  // statistics
  long long n_rounds = 0, job_rounds = 0, line_pairs = 0;
  int max_batch = 0;
  std::string init_err;
};

namespace {

void set_err(Job* j, int code, const std::string& m) {
  if (j->err == ECC_OK) {
    j->err = code;
    j->msg = m;
  }
}

std::string cuda_msg(const char* what, cudaError_t e) { return std::string(what) + ": " + cudaGetErrorString(e); }

// Allocation, input copies and precompute of one job on the admission stream.
bool admit_job(ecc_serve* S, Job* J) {
  const ecc_job& d = J->d;
  const Layout& L = J->L;
  cudaStream_t s = S->s_admit;
  cudaError_t e = cudaMallocAsync((void**)&J->dev, L.resident, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&J->tmp, L.transient, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_err(J, ECC_ENOMEM, cuda_msg("device allocation", e));
    return false;
  }
  const size_t n = (size_t)d.n_views;
  unsigned char* R = J->dev;
  unsigned char* T = J->tmp;
  cudaEventRecord(S->admit_t[0], s);
  e = cudaMemcpyAsync(R + L.P, d.P, n * 12 * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    if (d.motion0)
      e = cudaMemcpyAsync(R + L.theta0, d.motion0, n * 6 * sizeof(double), cudaMemcpyHostToDevice, s);
    else
      e = cudaMemsetAsync(R + L.theta0, 0, n * 6 * sizeof(double), s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(R + L.theta, R + L.theta0, n * 6 * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && d.motion_model == ECC_MOTION_AKIMA) {
    if (d.nodes0)
      e = cudaMemcpyAsync(R + L.nodes, d.nodes0, (size_t)d.n_nodes * 6 * sizeof(double), cudaMemcpyHostToDevice, s);
    else
      e = cudaMemsetAsync(R + L.nodes, 0, (size_t)d.n_nodes * 6 * sizeof(double), s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(R + L.status, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(T + L.images, d.images, n * (size_t)d.W * d.H * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    set_err(J, ECC_ECUDA, cuda_msg("input copy", e));
    return false;
  }
  cudaEventRecord(S->admit_t[1], s);
  ecc::view_setup_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(
      (int)n, (const double*)(R + L.P), nullptr, d.W, d.H, (ecc::ViewRec*)(R + L.views), (int*)(R + L.status));
  ecc::alpha_dir_kernel<<<(d.n_alpha + 255) / 256, 256, 0, s>>>(d.n_alpha, (float4*)(R + L.adir));
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    const ecc::LaunchHooks hk;
    e = ecc::launch_radon((const ecc::ViewRec*)(R + L.views), (int)n, (const float*)(T + L.images), d.W, d.H,
                          d.n_alpha, d.n_s, d.dtype, R + L.sino, (float*)(R + L.scales),
                          (ecc::RadonRow*)(T + L.rtable), T + L.wimg, (float*)(T + L.stage), L.batch, hk, s);
  }
  if (e != cudaSuccess) {
    set_err(J, ECC_ECUDA, cuda_msg("precompute launch", e));
    return false;
  }
  cudaEventRecord(S->admit_t[2], s);
  e = cudaFreeAsync(J->tmp, s);
  J->tmp = nullptr;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_err(J, ECC_ECUDA, cuda_msg("precompute", e));
    return false;
  }
  float up = 0.0f, pre = 0.0f;
  if (cudaEventElapsedTime(&up, S->admit_t[0], S->admit_t[1]) == cudaSuccess &&
      cudaEventElapsedTime(&pre, S->admit_t[1], S->admit_t[2]) == cudaSuccess) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->upload_ms += up;
    S->precompute_ms += pre;
  }
  return true;
}

void release_job_memory(ecc_serve* S, Job* J, cudaStream_t s) {
  if (J->tmp) cudaFreeAsync(J->tmp, s);
  if (J->dev) cudaFreeAsync(J->dev, s);
  J->tmp = nullptr;
  J->dev = nullptr;
  if (J->done) {
    cudaEventDestroy(J->done);
    J->done = nullptr;
  }
  if (J->slot >= 0) {
    S->free_slots.push_back(J->slot);
    J->slot = -1;
  }
}

void admission_loop(ecc_serve* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_admit.wait(lk, [&] {
      if (S->stop) return true;
      if (S->queue.empty()) return false;
      const Job* h = S->queue.front();
      return S->admitting + S->running < kMaxActive && !S->free_slots.empty() &&
             S->used + h->L.resident + h->L.transient <= S->budget;
    });
    if (S->stop) return;
    Job* J = S->queue.front();
    S->queue.pop_front();
    J->st = State::Admitting;
    J->t_admit = Clock::now();
    J->slot = S->free_slots.back();
    S->free_slots.pop_back();
    J->h_stage = reinterpret_cast<double*>(S->slots + (size_t)J->slot * kSlotBytes);
    S->used += J->L.resident + J->L.transient;
    ++S->admitting;
    lk.unlock();
    const bool ok = admit_job(S, J);
    lk.lock();
    --S->admitting;
    S->used -= J->L.transient;
    if (ok) {
      J->st = State::Active;
      ++S->running;
      S->ready.push_back(J);
      S->cv_round.notify_one();
    } else {
      cudaStreamSynchronize(S->s_admit);
      release_job_memory(S, J, S->s_admit);
      cudaStreamSynchronize(S->s_admit);
      S->used -= J->L.resident;
      J->st = State::Failed;
      J->t_done = Clock::now();
      S->cv_admit.notify_all();
    }
  }
}

// Copies the finished job's results to the caller and fills its result record.
void finish_job(ecc_serve* S, Job* J) {
  const ecc_job& d = J->d;
  const double* totals = J->h_stage;
  const double* theta = J->h_stage + (d.n_iters + 1);
  if (d.totals_out) std::memcpy(d.totals_out, totals, sizeof(double) * (d.n_iters + 1));
  if (d.motion_out) std::memcpy(d.motion_out, theta, sizeof(double) * 6 * d.n_views);
  if (d.motion_model == ECC_MOTION_AKIMA && d.nodes_out)
    std::memcpy(d.nodes_out, theta + 6 * d.n_views, sizeof(double) * 6 * d.n_nodes);
  J->t_done = Clock::now();
  ecc_result& r = J->res;
  const size_t nn = d.motion_model == ECC_MOTION_AKIMA ? (size_t)d.n_nodes : 0;
  std::memcpy(&r.flags, J->h_stage + (d.n_iters + 1) + 6 * d.n_views + 6 * nn, sizeof(int));
  r.iters = d.n_iters;
  r.total_first = totals[0];
  r.total_last = totals[d.n_iters];
  r.queue_ms = std::chrono::duration<double, std::milli>(J->t_admit - J->t_submit).count();
  r.latency_ms = std::chrono::duration<double, std::milli>(J->t_done - J->t_submit).count();
  r.footprint_bytes = J->L.resident + J->L.transient;
  const long long n = d.n_views;
  r.line_pairs = n * (n - 1) / 2 * (long long)d.n_kappa * (d.n_iters + 1);
  S->line_pairs += r.line_pairs;
  J->st = State::Done;
}

void round_loop(ecc_serve* S) {
  cudaSetDevice(S->device);
  std::vector<Job*> active, finishing;
  long long round = 0;
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    // completed jobs: results to the caller, memory back to the budget
    for (size_t i = 0; i < finishing.size();) {
      Job* J = finishing[i];
      const cudaError_t q = cudaEventQuery(J->done);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      if (q != cudaSuccess) set_err(J, ECC_ECUDA, cuda_msg("round", q));
      if (J->err == ECC_OK) {
        finish_job(S, J);
      } else {
        J->st = State::Failed;
        J->t_done = Clock::now();
      }
      release_job_memory(S, J, S->s_round);
      S->used -= J->L.resident;
      --S->running;
      finishing.erase(finishing.begin() + (long)i);
      S->cv_admit.notify_all();
    }
    for (Job* J : S->ready) active.push_back(J);
    S->ready.clear();
    if (active.empty()) {
      for (int b = 0; b < 2; ++b)  // no round in flight: account the last ones
        if (S->round_pending[b] && finishing.empty()) {
          float ms = 0.0f;
          if (cudaEventSynchronize(S->round_t1[b]) == cudaSuccess &&
              cudaEventElapsedTime(&ms, S->round_t0[b], S->round_t1[b]) == cudaSuccess)
            S->round_ms += ms;
          S->round_pending[b] = false;
        }
      if (S->stop && finishing.empty()) return;
      if (finishing.empty())
        S->cv_round.wait(lk, [&] { return S->stop || !S->ready.empty(); });
      else
        S->cv_round.wait_for(lk, std::chrono::microseconds(200));
      continue;
    }
    if (S->stop) {  // shutting down: drop the remaining work
      for (Job* J : active) {
        set_err(J, ECC_ECUDA, "context destroyed");
        J->st = State::Failed;
        finishing.push_back(J);
        if (!J->done) cudaEventCreateWithFlags(&J->done, cudaEventDisableTiming);
        cudaEventRecord(J->done, S->s_round);
      }
      active.clear();
      continue;
    }
    lk.unlock();
    // ---- one round over the active jobs
    const int b = (int)(round & 1);
    if (round >= 2) cudaEventSynchronize(S->round_ev[b]);  // the pinned copy of round - 2 is consumed
    if (S->round_pending[b]) {  // its timing events are complete too
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, S->round_t0[b], S->round_t1[b]) == cudaSuccess) {
        std::lock_guard<std::mutex> g(S->mu);
        S->round_ms += ms;
      }
      S->round_pending[b] = false;
    }
    const int nj = (int)active.size();
    ecc::ServeJob* H = S->h_jobs[b];
    long long* voff = S->h_off[b];
    long long* poff = voff + (kMaxActive + 1);
    long long* boff = poff + (kMaxActive + 1);
    voff[0] = poff[0] = boff[0] = 0;
    for (int i = 0; i < nj; ++i) {
      Job* J = active[i];
      const ecc_job& d = J->d;
      const Layout& L = J->L;
      unsigned char* R = J->dev;
      const long long n = d.n_views, np = n * (n - 1) / 2;
      ecc::ServeJob& s = H[i];
      s.pair.n_pairs = np;
      s.pair.prs = (const ecc::PairRec*)(R + L.prs);
      s.pair.ctile = (const float4*)(R + L.ctile);
      s.pair.n_tiles = (d.n_kappa + 31) / 32;
      s.pair.alpha_dir = (const float4*)(R + L.adir);
      s.pair.sino = R + L.sino;
      s.pair.scales = d.dtype == ECC_F16 ? (const float*)(R + L.scales) : nullptr;
      ecc::pair_args_grid(s.pair, d.n_alpha, d.n_s, d.W, d.H);
      s.pair.K = d.n_kappa;
      s.pair.cauchy_c = (float)d.cauchy_c;
      s.pair.per_pair = nullptr;
      s.pair.nk_out = nullptr;
      s.pair.block_partial = (double*)(R + L.partial);
      s.pair.Gpp = (double*)(R + L.Gpp);
      s.pair.status = (int*)(R + L.status);
      s.dtype = d.dtype;
      s.n_views = d.n_views;
      s.W = d.W;
      s.H = d.H;
      s.n_tiles = s.pair.n_tiles;
      s.do_grad = J->rounds < d.n_iters ? 1 : 0;
      s.step = d.step;
      s.P = (const double*)(R + L.P);
      s.theta = (double*)(R + L.theta);
      s.grad = (double*)(R + L.grad);
      s.views = (ecc::ViewRec*)(R + L.views);
      s.vtan = (ecc::ViewTan*)(R + L.vtan);
      s.gpp = (float2*)(R + L.gpp);
      s.total_out = (double*)(R + L.totals) + J->rounds;
      s.status = (int*)(R + L.status);
      s.model = d.motion_model;
      s.n_nodes = d.motion_model == ECC_MOTION_AKIMA ? d.n_nodes : 0;
      s.mask = d.param_mask ? d.param_mask : 0x3F;
      s.h = s.n_nodes > 1 ? (double)(d.n_views - 1) / (s.n_nodes - 1) : 1.0;
      s.theta0 = (const double*)(R + L.theta0);
      s.nodes = (double*)(R + L.nodes);
      s.jac = (double*)(R + L.jac);
      s.jbase = (int*)(R + L.jbase);
      voff[i + 1] = voff[i] + n;
      poff[i + 1] = poff[i] + np;
      boff[i + 1] = boff[i] + (np + kWarpsPerPairBlock - 1) / kWarpsPerPairBlock;
    }
    cudaStream_t s = S->s_round;
    ecc::ServeJob* dj = S->d_jobs + (size_t)b * kMaxActive;
    long long* dvoff = S->d_off + (size_t)b * 3 * (kMaxActive + 1);
    long long* dpoff = dvoff + (kMaxActive + 1);
    long long* dboff = dpoff + (kMaxActive + 1);
    cudaEventRecord(S->round_t0[b], s);
    cudaError_t e = cudaMemcpyAsync(dj, H, sizeof(ecc::ServeJob) * nj, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dvoff, voff, sizeof(long long) * 3 * (kMaxActive + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = ecc::launch_serve_motion(dj, dvoff, nj, voff[nj], s);
    if (e == cudaSuccess) e = ecc::launch_serve_setup(dj, dvoff, dpoff, nj, voff[nj], poff[nj], s);
    if (e == cudaSuccess) e = ecc::launch_serve_pairs(dj, dboff, nj, S->d_counter + b, S->pair_grid, s);
    if (e == cudaSuccess) e = ecc::launch_serve_grad(dj, dvoff, dpoff, nj, voff[nj], poff[nj], s);
    if (e == cudaSuccess) e = cudaEventRecord(S->round_t1[b], s);
    if (e == cudaSuccess) e = cudaEventRecord(S->round_ev[b], s);
    lk.lock();
    S->round_pending[b] = e == cudaSuccess;
    ++S->n_rounds;
    S->job_rounds += nj;
    S->max_batch = std::max(S->max_batch, nj);
    ++round;
    for (size_t i = 0; i < active.size();) {
      Job* J = active[i];
      ++J->rounds;
      if (e != cudaSuccess) set_err(J, ECC_ECUDA, cuda_msg("round launch", e));
      if (e != cudaSuccess || J->rounds > J->d.n_iters) {  // last evaluation issued: results to pinned memory
        const ecc_job& d = J->d;
        cudaMemcpyAsync(J->h_stage, J->dev + J->L.totals, sizeof(double) * (d.n_iters + 1), cudaMemcpyDeviceToHost,
                        s);
        cudaMemcpyAsync(J->h_stage + (d.n_iters + 1), J->dev + J->L.theta, sizeof(double) * 6 * d.n_views,
                        cudaMemcpyDeviceToHost, s);
        const size_t nn = d.motion_model == ECC_MOTION_AKIMA ? (size_t)d.n_nodes : 0;
        if (nn)
          cudaMemcpyAsync(J->h_stage + (d.n_iters + 1) + 6 * d.n_views, J->dev + J->L.nodes,
                          sizeof(double) * 6 * nn, cudaMemcpyDeviceToHost, s);
        // the job's device status word (ECC_STATUS_* bits), in the next double's slot
        cudaMemcpyAsync(J->h_stage + (d.n_iters + 1) + 6 * d.n_views + 6 * nn, J->dev + J->L.status, sizeof(int),
                        cudaMemcpyDeviceToHost, s);
        if (!J->done) cudaEventCreateWithFlags(&J->done, cudaEventDisableTiming);
        cudaEventRecord(J->done, s);
        J->st = State::Finishing;
        finishing.push_back(J);
        active.erase(active.begin() + (long)i);
        continue;
      }
      ++i;
    }
  }
}

int check_job(const ecc_job* j, std::string* why) {
  char b[256];
  auto bad = [&](const char* m) {
    *why = m;
    return ECC_EINVAL;
  };
  if (!j) return bad("job is NULL");
  if (!j->P || !j->images) return bad("job P or images is NULL");
  if (j->n_views < 2 || j->n_views > kMaxViewsServed) {
    std::snprintf(b, sizeof b, "n_views %d out of range [2, %d]", j->n_views, kMaxViewsServed);
    return bad(b);
  }
  if (j->W < 2 || j->H < 2 || j->W > 16384 || j->H > 16384) return bad("detector size out of range");
  if (j->n_alpha < 4 || j->n_alpha > 65535 || j->n_s < 2 || j->n_s > 65535) return bad("sinogram grid out of range");
  if (j->dtype != ECC_F32 && j->dtype != ECC_F16 && j->dtype != ECC_BF16) return bad("unknown dtype");
  if (j->n_kappa < 1 || j->n_kappa > 65536) return bad("n_kappa out of range [1, 65536]");
  if (j->n_iters < 0 || j->n_iters > kMaxIters) return bad("n_iters out of range");
  if (!std::isfinite(j->step) || !std::isfinite(j->cauchy_c)) return bad("step or cauchy_c is not finite");
  if (j->motion_model != ECC_MOTION_PER_VIEW && j->motion_model != ECC_MOTION_AKIMA) return bad("unknown motion_model");
  if (j->motion_model == ECC_MOTION_AKIMA && (j->n_nodes < 3 || j->n_nodes > j->n_views))
    return bad("n_nodes out of range [3, n_views] for the Akima motion model");
  if (j->param_mask < 0 || j->param_mask > 0x3F) return bad("param_mask has bits beyond the six parameters");
  const size_t nn = j->motion_model == ECC_MOTION_AKIMA ? (size_t)j->n_nodes : 0;
  if (sizeof(double) * ((size_t)j->n_iters + 2 + 6 * (size_t)j->n_views + 6 * nn) > kSlotBytes)
    return bad("n_iters + 6 n_views + 6 n_nodes too large for the result staging");
  // the geometry is small enough to check on the host; the images are checked on the
  // device (a non-finite sinogram value drops the pairs it reaches, see ecc_result.flags)
  auto all_finite = [](const double* x, size_t n) {
    for (size_t i = 0; i < n; ++i)
      if (!std::isfinite(x[i])) return false;
    return true;
  };
  if (!all_finite(j->P, 12 * (size_t)j->n_views)) return bad("P has a non-finite entry");
  if (j->motion0 && !all_finite(j->motion0, 6 * (size_t)j->n_views)) return bad("motion0 has a non-finite entry");
  if (nn && j->nodes0 && !all_finite(j->nodes0, 6 * nn)) return bad("nodes0 has a non-finite entry");
  return ECC_OK;
}

}  // namespace

namespace ecc {

int serve_footprint(const ecc_job* job, size_t* bytes, std::string* why) {
  const int rc = check_job(job, why);
  if (rc != ECC_OK) return rc;
  const Layout L = layout_of(*job);
  *bytes = L.resident + L.transient;
  return ECC_OK;
}

ecc_serve* serve_create(int device, size_t budget, std::string* why) {
  ecc_serve* S = new ecc_serve();
  S->device = device;
  cudaError_t e = cudaSetDevice(device);
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  S->budget = budget ? budget : free_b / 10 * 8;  // no context bound: 80 % of the free memory now
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_admit, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_round, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&S->d_jobs, sizeof(ServeJob) * 2 * kMaxActive);
  if (e == cudaSuccess) e = cudaMalloc(&S->d_off, sizeof(long long) * 2 * 3 * (kMaxActive + 1));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_counter, sizeof(unsigned long long) * 2);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMallocHost(&S->h_jobs[b], sizeof(ServeJob) * kMaxActive);
    if (e == cudaSuccess) e = cudaMallocHost(&S->h_off[b], sizeof(long long) * 3 * (kMaxActive + 1));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->round_ev[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&S->round_t0[b]);
    if (e == cudaSuccess) e = cudaEventCreate(&S->round_t1[b]);
  }
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventCreate(&S->admit_t[k]);
  if (e == cudaSuccess) e = cudaMallocHost(&S->slots, kSlotBytes * kMaxActive);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *why = cuda_msg("serving set-up", e);
    serve_destroy(S);
    return nullptr;
  }
  S->pair_grid = sms * serve_pairs_blocks_per_sm();
  for (int i = kMaxActive - 1; i >= 0; --i) S->free_slots.push_back(i);
  S->th_admit = std::thread(admission_loop, S);
  S->th_round = std::thread(round_loop, S);
  return S;
}

void serve_destroy(ecc_serve* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_admit.notify_all();
  S->cv_round.notify_all();
  if (S->th_admit.joinable()) S->th_admit.join();
  if (S->th_round.joinable()) S->th_round.join();
  cudaSetDevice(S->device);
  if (S->s_round) cudaStreamSynchronize(S->s_round);
  if (S->s_admit) cudaStreamSynchronize(S->s_admit);
  for (auto& kv : S->jobs) {
    Job* J = kv.second;
    release_job_memory(S, J, S->s_round ? S->s_round : 0);
    delete J;
  }
  if (S->s_round) cudaStreamSynchronize(S->s_round);
  if (S->d_jobs) cudaFree(S->d_jobs);
  if (S->d_off) cudaFree(S->d_off);
  if (S->d_counter) cudaFree(S->d_counter);
  for (int b = 0; b < 2; ++b) {
    if (S->h_jobs[b]) cudaFreeHost(S->h_jobs[b]);
    if (S->h_off[b]) cudaFreeHost(S->h_off[b]);
    if (S->round_ev[b]) cudaEventDestroy(S->round_ev[b]);
    if (S->round_t0[b]) cudaEventDestroy(S->round_t0[b]);
    if (S->round_t1[b]) cudaEventDestroy(S->round_t1[b]);
  }
  for (int k = 0; k < 3; ++k)
    if (S->admit_t[k]) cudaEventDestroy(S->admit_t[k]);
  if (S->slots) cudaFreeHost(S->slots);
  if (S->s_admit) cudaStreamDestroy(S->s_admit);
  if (S->s_round) cudaStreamDestroy(S->s_round);
  delete S;
}

int serve_submit(ecc_serve* S, const ecc_job* job, uint64_t* ticket, std::string* why) {
  if (!ticket) {
    *why = "ticket is NULL";
    return ECC_EINVAL;
  }
  int rc = check_job(job, why);
  if (rc != ECC_OK) return rc;
  Job* J = new Job();
  J->d = *job;
  J->L = layout_of(*job);
  if (J->L.resident + J->L.transient > S->budget) {
    char b[256];
    std::snprintf(b, sizeof b, "job needs %zu bytes of device memory, the serving budget is %zu",
                  J->L.resident + J->L.transient, S->budget);
    *why = b;
    delete J;
    return ECC_EADMIT;
  }
  J->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    J->ticket = S->next_ticket++;
    S->jobs[J->ticket] = J;
    S->queue.push_back(J);
  }
  S->cv_admit.notify_one();
  *ticket = J->ticket;
  return ECC_OK;
}

int serve_poll(ecc_serve* S, uint64_t ticket, ecc_result* out, std::string* why) {
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) {
    *why = "unknown ticket";
    return ECC_EINVAL;
  }
  Job* J = it->second;
  if (J->st != State::Done && J->st != State::Failed) return ECC_EPENDING;
  ecc_result r = J->res;
  r.status = J->st == State::Done ? ECC_OK : J->err;
  if (J->st == State::Failed) {
    r.queue_ms = std::chrono::duration<double, std::milli>(J->t_admit - J->t_submit).count();
    r.latency_ms = std::chrono::duration<double, std::milli>(J->t_done - J->t_submit).count();
    *why = J->msg;
  }
  if (out) *out = r;
  S->jobs.erase(it);
  delete J;
  return r.status;
}

void serve_times(ecc_serve* S, double* upload_ms, double* precompute_ms, double* round_ms) {
  std::lock_guard<std::mutex> lk(S->mu);
  if (upload_ms) *upload_ms = S->upload_ms;
  if (precompute_ms) *precompute_ms = S->precompute_ms;
  if (round_ms) *round_ms = S->round_ms;
}

void serve_stats(ecc_serve* S, long long* rounds, long long* job_rounds, int* max_batch, long long* line_pairs) {
  std::lock_guard<std::mutex> lk(S->mu);
  if (rounds) *rounds = S->n_rounds;
  if (job_rounds) *job_rounds = S->job_rounds;
  if (max_batch) *max_batch = S->max_batch;
  if (line_pairs) *line_pairs = S->line_pairs;
}

}  // namespace ecc

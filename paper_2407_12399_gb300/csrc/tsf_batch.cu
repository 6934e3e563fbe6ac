// tsf_batch.cu -- many independent fields solved together.  Each field has
// its own non-blocking stream and is driven by one host thread of a small
// pool, so the fields' kernels (most stages use a fraction of the GPU) run
// concurrently.  Every field's iteration is exactly tsf_solver_step /
// tsf_simplify on that field: a field's trajectory does not depend on the
// batch it is in.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/tsf.h"
#include "tsf_kernels.cuh"

namespace tsf {
int full_diagram_for_tuning(tsf_field* F);
}

struct tsf_batch {
  int device = 0;  // current when the batch was created; the workers use it too
  std::vector<tsf_field*> fields;
  std::vector<cudaStream_t> streams;
  // worker pool: run(job) calls job(i) for every field index, spread over
  // the workers, and returns when all are done
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::function<void(int)> job;
  long long generation = 0;
  int pending = 0;
  bool stop = false;

  void worker(int w, int nw) {
    cudaSetDevice(device);  // the current device is per host thread
    long long seen = 0;
    for (;;) {
      std::function<void(int)> j;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || generation != seen; });
        if (stop) return;
        seen = generation;
        j = job;
      }
      for (int i = w; i < (int)fields.size(); i += nw) j(i);
      {
        std::lock_guard<std::mutex> lk(mu);
        if (--pending == 0) cv_done.notify_all();
      }
    }
  }

  void run(std::function<void(int)> f) {
    std::unique_lock<std::mutex> lk(mu);
    job = std::move(f);
    pending = (int)workers.size();
    ++generation;
    cv_work.notify_all();
    cv_done.wait(lk, [&] { return pending == 0; });
  }

  ~tsf_batch() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv_work.notify_all();
    for (auto& t : workers) t.join();
    for (auto* f : fields) tsf_destroy_field(f);
    for (auto s : streams)
      if (s) cudaStreamDestroy(s);
  }
};

namespace {

int first_error(const std::vector<int>& codes) {
  for (int c : codes)
    if (c != TSF_OK) return c;
  return TSF_OK;
}

}  // namespace

extern "C" {

int tsf_batch_create(int n, const int* lx, const int* ly, const int* lz, const float* const* values,
                     int values_on_device, tsf_batch** out) {
  if (!out || n <= 0 || !lx || !ly || !lz || !values) return TSF_EINVAL;
  *out = nullptr;
  tsf_batch* b = nullptr;
  try {
    b = new tsf_batch();
  } catch (...) {
    return TSF_ENOMEM;
  }
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return TSF_ECUDA;
  }
  for (int i = 0; i < n; ++i) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return TSF_ECUDA;
    }
    b->streams.push_back(s);
    tsf_field* f = nullptr;
    int r = tsf_create_field(lx[i], ly[i], lz[i], values[i], values_on_device, s, &f);
    if (r != TSF_OK) {
      delete b;
      return r;
    }
    b->fields.push_back(f);
  }
  unsigned hw = std::thread::hardware_concurrency();
  int nw = std::max(1, std::min(n, (int)std::max(2u, hw)));
  try {
    for (int w = 0; w < nw; ++w) b->workers.emplace_back([b, w, nw] { b->worker(w, nw); });
  } catch (...) {
    delete b;
    return TSF_ENOMEM;
  }
  *out = b;
  return TSF_OK;
}

int tsf_batch_destroy(tsf_batch* b) {
  delete b;
  return TSF_OK;
}

int tsf_batch_size(const tsf_batch* b) { return b ? (int)b->fields.size() : 0; }

int tsf_batch_field(tsf_batch* b, int i, tsf_field** out) {
  if (!b || !out || i < 0 || i >= (int)b->fields.size()) return TSF_EINVAL;
  *out = b->fields[i];
  return TSF_OK;
}

int tsf_batch_set_signal_thresholds(tsf_batch* b, const float* fractions) {
  if (!b || !fractions) return TSF_EINVAL;
  std::vector<int> codes(b->fields.size(), TSF_OK);
  b->run([&](int i) { codes[i] = tsf_set_signal_threshold(b->fields[i], fractions[i]); });
  return first_error(codes);
}

int tsf_batch_step(tsf_batch* b, const tsf_params* params, tsf_stats* stats) {
  if (!b || !params) return TSF_EINVAL;
  std::vector<int> codes(b->fields.size(), TSF_OK);
  b->run([&](int i) { codes[i] = tsf_solver_step(b->fields[i], params, stats ? stats + i : nullptr); });
  return first_error(codes);
}

int tsf_batch_autotune(tsf_batch* b, int* choice, double* ms, int cap) {
  if (!b || !choice || cap < 0 || (cap > 0 && !ms)) return TSF_EINVAL;
  // candidates: the D1 Morse boundaries' first phase (knob 7): half a warp
  // per column with 64 + 128 frontier and stage entries, half a warp with
  // 32 + 64, a quarter of a warp with 16 + 32, one warp with 64 + 128
  constexpr int kCand = 4;
  constexpr int64_t kKnob[kCand] = {7, 5, 6, 4};
  const int64_t keep = tsf::get_knob(7);
  double best = -1.0;
  int arg = 0;
  for (int c = 0; c < kCand; ++c) {
    tsf::set_knob(7, kKnob[c]);
    double t = 0.0;
    for (int rep = 0; rep < 2; ++rep) {  // the first pass sizes buffers; the second is timed
      std::vector<int> codes(b->fields.size(), TSF_OK);
      const auto t0 = std::chrono::steady_clock::now();
      b->run([&](int i) { codes[i] = tsf::full_diagram_for_tuning(b->fields[i]); });
      t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      const int r = first_error(codes);
      if (r != TSF_OK) {
        tsf::set_knob(7, keep);
        return r;
      }
    }
    if (c < cap) ms[c] = t;
    if (best < 0.0 || t < best) {
      best = t;
      arg = c;
    }
  }
  tsf::set_knob(7, kKnob[arg]);
  *choice = arg;
  return TSF_OK;
}

int tsf_batch_simplify(tsf_batch* b, const tsf_params* params, tsf_stats* stats) {
  if (!b || !params) return TSF_EINVAL;
  std::vector<int> codes(b->fields.size(), TSF_OK);
  b->run([&](int i) {
    codes[i] = tsf_simplify(b->fields[i], params, nullptr, 0, stats ? stats + i : nullptr);
  });
  return first_error(codes);
}

}  // extern "C"

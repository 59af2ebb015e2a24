// Launch counter and per-phase CUDA-event profiler used by the benchmark.
#include <atomic>
#include <cstring>
#include <vector>

#include "common.h"

namespace vb {
namespace {
std::atomic<unsigned long long> g_launches{0};
struct Pending {
  int phase;
  cudaEvent_t a, b;
};
// Calls of a phase are numbered in order; with every = k > 1 only calls
// whose number is a multiple of k get events (systematic sampling: every
// stretch of k consecutive calls contributes one), and the phase's time is
// the sampled time scaled by calls / sampled calls. Call counts and flops
// are exact.
struct Prof {
  int every = 0;
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> open_start;  // per phase
  unsigned long long seq[PH_COUNT] = {0};
  double ms[PH_COUNT] = {0};
  long long calls[PH_COUNT] = {0};
  long long sampled[PH_COUNT] = {0};
  double pflops[PH_COUNT] = {0};
  double pbytes[PH_COUNT] = {0};
  double flops[2] = {0, 0};
  double krylov_flops = 0;
} g_prof;

cudaEvent_t take_event() {
  if (!g_prof.pool.empty()) {
    cudaEvent_t e = g_prof.pool.back();
    g_prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool prof_on() { return g_prof.every > 0; }

void prof_begin(int phase, cudaStream_t st) {
  if (!g_prof.every) return;
  if (g_prof.open_start.size() < PH_COUNT) g_prof.open_start.assign(PH_COUNT, nullptr);
  g_prof.calls[phase]++;
  if (g_prof.seq[phase]++ % (unsigned long long)g_prof.every != 0) {
    g_prof.open_start[phase] = nullptr;
    return;
  }
  cudaEvent_t e = take_event();
  cudaEventRecord(e, st);
  g_prof.open_start[phase] = e;
}

void prof_end(int phase, cudaStream_t st, double flops, double bytes) {
  if (!g_prof.every) return;
  g_prof.pflops[phase] += flops;
  g_prof.pbytes[phase] += bytes;
  if (phase < 2) g_prof.flops[phase] += flops;
  if (phase == PH_KRYLOV) g_prof.krylov_flops += flops;
  if (g_prof.open_start.size() < PH_COUNT || !g_prof.open_start[phase]) return;
  cudaEvent_t e = take_event();
  cudaEventRecord(e, st);
  g_prof.pending.push_back(Pending{phase, g_prof.open_start[phase], e});
  g_prof.open_start[phase] = nullptr;
}

void prof_note(int phase, double v) {
  if (g_prof.every && phase >= 0 && phase < PH_COUNT) g_prof.pflops[phase] += v;
}

void prof_collect() {
  if (g_prof.pending.empty()) return;
  std::vector<Pending> keep;
  for (const Pending &p : g_prof.pending) {
    if (cudaEventQuery(p.b) != cudaSuccess) {
      cudaGetLastError();
      keep.push_back(p);
      continue;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    g_prof.ms[p.phase] += ms;
    g_prof.sampled[p.phase] += 1;
    g_prof.pool.push_back(p.a);
    g_prof.pool.push_back(p.b);
  }
  g_prof.pending.swap(keep);
}

}  // namespace vb

extern "C" {

unsigned long long vb_kernel_launches(void) { return vb::g_launches.load(); }

vb_status vb_profile_enable(int every) {
  if (every < 0) return vb::fail(VB_EINVAL, "vb_profile_enable: negative sampling interval");
  vb::g_prof.every = every;
  return VB_OK;
}

vb_status vb_profile_read(vb_profile *out, int reset) {
  if (!out) return vb::fail(VB_EINVAL, "vb_profile_read: null argument");
  vb::prof_collect();
  std::memset(out, 0, sizeof(*out));
  for (int i = 0; i < vb::PH_COUNT; ++i) {
    const long long c = vb::g_prof.calls[i], k = vb::g_prof.sampled[i];
    out->ms[i] = k > 0 ? vb::g_prof.ms[i] * ((double)c / (double)k) : 0.0;
    out->calls[i] = c;
    out->flops[i] = vb::g_prof.pflops[i];
    out->bytes[i] = vb::g_prof.pbytes[i];
  }
  out->heff_flops[0] = vb::g_prof.flops[0];
  out->heff_flops[1] = vb::g_prof.flops[1];
  out->krylov_flops = vb::g_prof.krylov_flops;
  if (reset) {
    for (int i = 0; i < vb::PH_COUNT; ++i) {
      vb::g_prof.ms[i] = 0;
      vb::g_prof.calls[i] = 0;
      vb::g_prof.sampled[i] = 0;
      vb::g_prof.seq[i] = 0;
      vb::g_prof.pflops[i] = 0;
      vb::g_prof.pbytes[i] = 0;
    }
    vb::g_prof.flops[0] = vb::g_prof.flops[1] = 0;
    vb::g_prof.krylov_flops = 0;
  }
  return VB_OK;
}

}  // extern "C"

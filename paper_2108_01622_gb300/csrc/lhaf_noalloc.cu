// Allocation-free loop hafnian: the same sieve kernels as lhaf(), with their scratch memory in a
// fixed device array of this file instead of a context workspace.
//
// Who needs this: callers that must not call cudaMalloc/cudaFree at all, for example code running
// where another allocator (a framework's caching allocator, a pre-reserved memory pool) owns the
// device memory and a raw cudaMalloc could fail or fragment it, or latency-critical loops where
// the implicit device synchronisation of cudaMalloc/cudaFree is not acceptable. lhaf_ctx_create
// allocates a workspace; this entry point needs no context and allocates nothing.
//
// The scratch array below is a file-scope device variable: every GPU that loads the library holds
// it (224 KiB) until the process exits. In host code its name is only a host-side stand-in for the
// device variable, never a usable device address, so the device address is looked up once per
// device with cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "../../include/lhaf.h"
#include "lhaf_internal.h"
#include "lhaf_plan.h"
#include "lhaf_ctx.h"

namespace {

using namespace lhafgpu;

// Scratch limits: slot matrix for working dimension <= kMaxDim in FP64 and FP32, plus one
// double-double partial (4 doubles) for each of at most kNoAllocTeams teams.
constexpr int kNoAllocTeams = 4096;
constexpr size_t kChatBytes = (size_t)kMaxDim * kMaxDim * sizeof(double2);     // 64 KiB
constexpr size_t kChat32Bytes = (size_t)kMaxDim * kMaxDim * sizeof(float2);    // 32 KiB
constexpr size_t kPartialBytes = (size_t)kNoAllocTeams * 4 * sizeof(double);   // 128 KiB
constexpr size_t kScratchBytes = kChatBytes + kChat32Bytes + kPartialBytes;    // 224 KiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current). Looked up with
// cudaGetSymbolAddress on every call made outside stream capture (so a module reloaded after
// cudaDeviceReset is found again) and cached per device; a call made while `stream` is capturing
// uses the cached address (the first call on a device should come before any capture).
lhaf_status scratch_address(int device, cudaStream_t stream, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return LHAF_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;  // cannot tell: do not touch the module state
  }
  if (cs == cudaStreamCaptureStatusNone || !g_scratch_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LHAF_ECUDA;
    }
    g_scratch_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[device]);
  return LHAF_OK;
}

__global__ void write_one(double2* out) { *out = make_double2(1.0, 0.0); }

int pick_team(bool fp32, const Plan& pl, int* occ_out) {
  const char* env = std::getenv("LHAF_TEAM");
  const int forced = env ? std::atoi(env) : 0;
  const int cands[5] = {8, 16, 32, 64, 128};
  double best = -1.0;
  int best_g = 0, best_occ = 0;
  for (int g : cands) {
    if (forced && g != forced) continue;
    const size_t smem = cta_shared_bytes(fp32, g, pl.nd, pl.H, pl.Hl, pl.P);
    if (smem > 227 * 1024) continue;
    const int occ = max_ctas_per_sm(fp32, g, smem);
    if (occ <= 0) continue;
    const double warps = (double)occ * cta_threads(g) / 32.0;
    const double score = model_lane_efficiency(pl.nd, pl.Hl, pl.h, pl.bord, g) * std::min(1.0, warps / 4.0) *
                         (warps >= 8.0 ? 1.0 : 0.9);
    if (score > best) {
      best = score;
      best_g = g;
      best_occ = occ;
    }
  }
  *occ_out = best_occ;
  return best_g;
}

}  // namespace

extern "C" lhaf_status lhaf_noalloc(int device, void* cuda_stream, int M, const lhaf_c128* B,
                                    const lhaf_c128* gamma, const int32_t* reps, uint32_t flags,
                                    lhaf_c128* out) {
  if (M <= 0 || !B || !out) return LHAF_EINVAL;
  if (flags & LHAF_ET) return LHAF_EINVAL;  // the finite difference sieve only
  if (flags & LHAF_DEVICE_PTRS) flags &= ~LHAF_DEVICE_PTRS;  // always device pointers here
  const bool fp32 = (flags & LHAF_FP32_TERMS) != 0;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return LHAF_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return LHAF_ECUDA;
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};

  Plan pl;
  const bool loops = !(flags & LHAF_NO_LOOPS);
  lhaf_status st = build_plan(M, reps, flags, loops, pl);
  if (st != LHAF_OK) return st;  // includes LHAF_ETOOBIG for n_dim > 64 (the slot-matrix limit)
  if (pl.nd > kMaxDim) return LHAF_ETOOBIG;
  if (fp32 && pl.h > kFp32MaxDegree) return LHAF_ETOOBIG;  // FP32 terms beyond their stated bound

  if (pl.N == 0) {  // lhaf of the empty pattern is 1
    write_one<<<1, 1, 0, stream>>>((double2*)out);
    return cudaGetLastError() == cudaSuccess ? LHAF_OK : LHAF_ECUDA;
  }

  unsigned char* base = nullptr;
  st = scratch_address(device, stream, &base);
  if (st != LHAF_OK) return st;
  double2* chat = reinterpret_cast<double2*>(base);
  float2* chat32 = reinterpret_cast<float2*>(base + kChatBytes);
  double* partials = reinterpret_cast<double*>(base + kChatBytes + kChat32Bytes);

  int occ = 0;
  const int team = pick_team(fp32, pl, &occ);
  if (team == 0) return LHAF_ETOOBIG;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return LHAF_ECUDA;

  TermParams p;
  fill_params(pl, fp32, false, team, flags, p);  // the whole sieve on the full working matrix
  // Grid: at most one resident wave, and never more teams than the scratch holds partials for.
  const int tpc = teams_per_cta(team);
  uint64_t grid = (pl.T + tpc - 1) / tpc;
  grid = std::min<uint64_t>(grid, (uint64_t)sms * (uint64_t)occ);
  grid = std::min<uint64_t>(grid, (uint64_t)(kNoAllocTeams / tpc));
  if (grid < 1) grid = 1;
  p.total_teams = grid * (uint64_t)tpc;
  p.rounds = (pl.T + p.total_teams - 1) / p.total_teams;
  p.t_begin = 0;
  p.t_end = pl.T;

  // Nothing in the scratch has to start at zero: the gather writes every slot-matrix entry the
  // term kernel reads, every launched team writes its partial, and the reduction reads exactly
  // the partials of this launch.
  if (launch_gather((const double2*)B, (const double2*)gamma, M, pl.slot_mode.data(), pl.P, pl.bord, chat,
                    fp32 ? chat32 : nullptr, stream) != cudaSuccess)
    return LHAF_ECUDA;
  const void* chat_arg = fp32 ? (const void*)chat32 : (const void*)chat;
  if (launch_terms(fp32, team, chat_arg, p, (int)grid, partials, stream) != cudaSuccess) return LHAF_ECUDA;
  if (launch_reduce(partials, (long long)p.total_teams, pl.h, nullptr, (double2*)out, stream) != cudaSuccess)
    return LHAF_ECUDA;
  return LHAF_OK;
}

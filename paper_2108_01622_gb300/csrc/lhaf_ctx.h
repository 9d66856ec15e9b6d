// The library context: device, stream, workspace, autotuning cache (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/lhaf.h"
#include "lhaf_internal.h"
#include "lhaf_plan.h"

// Device buffer that only grows (cudaMalloc on growth).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  bool reserve(size_t n) {
    if (n <= bytes) return true;
    cudaFree(p);
    p = nullptr;
    bytes = 0;
    if (cudaMalloc(&p, n) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    bytes = n;
    return true;
  }
  void release() {
    cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

// Pinned host buffer that only grows.
struct HostBuf {
  void* p = nullptr;
  size_t bytes = 0;
  bool reserve(size_t n) {
    if (n <= bytes) return true;
    cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    if (cudaMallocHost(&p, n) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    bytes = n;
    return true;
  }
  void release() {
    cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
  }
};

// Autotuning key: precision, staged series, working dimension, La Budde truncation, degree,
// border, and the kernel family (0 = single loop hafnian, 1 = batched).
using TuneKey = std::tuple<int, int, int, int, int, int, int>;

struct lhaf_ctx {
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // device workspace
  double2* d_chat = nullptr;
  float2* d_chat32 = nullptr;
  double* d_partials = nullptr;
  size_t partial_cap = 0;  // teams
  double* d_out = nullptr;  // 4 dd doubles + 2 value doubles
  void* d_stage = nullptr;  // staged characteristic polynomials (series_kernel input)
  double* d_wstage = nullptr;
  size_t stage_bytes = 0, wstage_terms = 0;
  // pinned host staging
  double2* h_chat = nullptr;
  float2* h_chat32 = nullptr;
  double* h_out = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, tev0 = nullptr, tev1 = nullptr;
  // batched form
  DevBuf b_items, b_units, b_queue, b_next, b_partials, b_unit_begin, b_item_h, b_chat, b_chat32, b_out,
      b_stage, b_wstage, b_gpart, b_gout;
  HostBuf hb_items, hb_units, hb_queue, hb_unit_begin, hb_item_h, hb_chat, hb_chat32, hb_out, hb_gout;
  // measured best team size per problem shape
  std::map<TuneKey, int> tuned;
  std::mutex mu;
};

namespace lhafgpu {
// Team size for a problem shape: LHAF_TEAM forces one; otherwise the fastest candidate on a short
// timed slice of real terms (chat must already be on the device), cached in ctx->tuned.
int pick_team(lhaf_ctx* ctx, bool fp32, const Plan& pl, bool staged, int family, const void* chat,
              int* ctas_per_sm);
// Fill the sieve description of a plan (everything but the term range and the grid).
void fill_params(const Plan& pl, bool fp32, bool staged, int team, uint32_t flags, TermParams& p);
}  // namespace lhafgpu

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

// Buffers of one grouped evaluation: the sieves (items, or their zero-digit groups) of one loop
// hafnian (ctx->gw) or of a batch (ctx->bw, or a batched plan's own, whose captured graph holds
// these addresses).
struct BatchWork {
  DevBuf items;      // sieve descriptors (BatchItem)
  DevBuf chunks;     // chunk offsets per sieve (long long), class after class
  DevBuf seg_begin;  // per launch: entry offsets of its item segments (long long)
  DevBuf seg_item;   // per launch: the item of each segment (int)
  DevBuf item_h, acc, entries, chat, chat32, out, stage, wstage, in_B, in_gamma;
  DevBuf counter;    // chunk queue of a grouped launch (zeroed before each launch)
  DevBuf et_table;   // eigenvalue-trace rank table of one loop hafnian
  DevBuf parts;      // per-chunk dd partials of an unstaged launch (4 doubles per chunk term slot)
  HostBuf h_et_table;
  HostBuf h_items, h_chunks, h_seg_begin, h_seg_item, h_item_h, h_chat, h_chat32, h_out, h_in;
  cudaEvent_t uploaded = nullptr;  // after the last copies that read the pinned buffers above
  void release() {
    if (uploaded) cudaEventDestroy(uploaded);
    uploaded = nullptr;
    for (DevBuf* b : {&items, &chunks, &seg_begin, &seg_item, &item_h, &acc, &entries, &chat, &chat32, &out, &stage,
                      &wstage, &in_B, &in_gamma, &counter, &et_table, &parts})
      b->release();
    for (HostBuf* b : {&h_et_table, &h_items, &h_chunks, &h_seg_begin, &h_seg_item, &h_item_h, &h_chat, &h_chat32, &h_out, &h_in})
      b->release();
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
  // batched form and adjoint
  BatchWork bw;
  BatchWork gw;  // one loop hafnian's zero-digit groups (descriptors in items, chunk offsets in units)
  DevBuf b_gpart, b_gout;
  HostBuf hb_gout;
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
int ctas_per_sm_override(int occ);
// Grow the context's staging buffer (synchronising its stream first) to at least `bytes` of
// coefficient rows and `terms` weights; false (and no buffer) if the allocation fails.
bool ensure_stage(lhaf_ctx* ctx, size_t bytes, size_t terms);

uint64_t balanced_grid(uint64_t n, int tpc, uint64_t max_ctas, unsigned long long* rounds);
}  // namespace lhafgpu

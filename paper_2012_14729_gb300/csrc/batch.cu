// Batched step: many independent domains of uneven sizes and force forms
// advance together, one persistent launch per time step.  The CTAs take
// (instance, tile) items of a work-list sorted by force form from a ticket
// counter (the next unclaimed item goes to whichever CTA asks first, so that
// the CTAs finish together although items differ in cost); each item runs
// the same per-tile passes as the single-domain kernels, with the instance's
// arguments taken from a table in global memory (FP32 storage).  Gather-mode
// batches run tiles of kTY or kShortRows rows (two or one collision nodes
// per thread); the autotuner times both.
#include "step_kernel.cuh"

namespace pflbm {

namespace {

// shared memory of the largest form
constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int kFieldsMax =
    cmax(cmax(cmax(Fields<kSTF1>::BYTES, Fields<kSTF2>::BYTES),
              cmax(Fields<kCPF1>::BYTES, Fields<kCPF2>::BYTES)),
         cmax(cmax(Fields<kPF1>::BYTES, Fields<kPF2>::BYTES),
              cmax(Fields<kCSF1>::BYTES, Fields<kCSF2>::BYTES)));
constexpr int kArgsBytes = pad128((int)sizeof(StepArgs));

template <class ST, int NT, bool INNER, int TY>
__device__ __forceinline__ void gather_item(const StepArgs& a, int form, unsigned char* fs, int x0,
                                            int y0) {
  using S = GatherSrc<ST, INNER>;
  const S src{};
  switch (form) {
    case kSTF1: step_tile<kSTF1, ST, NT, S, false, TY, false, false>(a, src, fs, x0, y0); break;
    case kSTF2: step_tile<kSTF2, ST, NT, S, false, TY, false, false>(a, src, fs, x0, y0); break;
    case kCPF1: step_tile<kCPF1, ST, NT, S, false, TY, false, false>(a, src, fs, x0, y0); break;
    case kCPF2: step_tile<kCPF2, ST, NT, S, false, TY, false, false>(a, src, fs, x0, y0); break;
    case kPF1: step_tile<kPF1, ST, NT, S, false, TY, false, false>(a, src, fs, x0, y0); break;
    case kPF2: step_tile<kPF2, ST, NT, S, false, TY, false, false>(a, src, fs, x0, y0); break;
    case kCSF1: step_tile<kCSF1, ST, NT, S, false, TY, false, false>(a, src, fs, x0, y0); break;
    default: step_tile<kCSF2, ST, NT, S, false, TY, false, false>(a, src, fs, x0, y0); break;
  }
}

template <class ST, int MODE, int NT, int TY>
__device__ __forceinline__ void run_item(const StepArgs& a, const StepArgs& ga, int form,
                                         unsigned char* bx, unsigned char* fs, int x0, int y0) {
  if constexpr (MODE == kBoxes) {
    static_assert(TY == kTY, "box staging is laid out for full tiles");
    const BoxSrc<ST> src{bx};
    switch (form) {
      case kSTF1: step_tile<kSTF1, ST, NT, BoxSrc<ST>, false, kTY, false, false>(a, src, fs, x0, y0); break;
      case kSTF2: step_tile<kSTF2, ST, NT, BoxSrc<ST>, false, kTY, false, false>(a, src, fs, x0, y0); break;
      case kCPF1: step_tile<kCPF1, ST, NT, BoxSrc<ST>, false, kTY, false, false>(a, src, fs, x0, y0); break;
      case kCPF2: step_tile<kCPF2, ST, NT, BoxSrc<ST>, false, kTY, false, false>(a, src, fs, x0, y0); break;
      case kPF1: step_tile<kPF1, ST, NT, BoxSrc<ST>, false, kTY, false, false>(a, src, fs, x0, y0); break;
      case kPF2: step_tile<kPF2, ST, NT, BoxSrc<ST>, false, kTY, false, false>(a, src, fs, x0, y0); break;
      case kCSF1: step_tile<kCSF1, ST, NT, BoxSrc<ST>, false, kTY, false, false>(a, src, fs, x0, y0); break;
      default: step_tile<kCSF2, ST, NT, BoxSrc<ST>, false, kTY, false, false>(a, src, fs, x0, y0); break;
    }
  } else if (inner_tile<TY>(a.L, x0, y0)) {
    gather_item<ST, NT, true, TY>(a, form, fs, x0, y0);
  } else {
    gather_item<ST, NT, false, TY>(a, form, fs, x0, y0);
  }
}

// table: 2 entries per instance (parity p reads buffer cur ^ p); items:
// (instance, x0, y0, form).  The step parity `bp` selects the entries.
template <int MODE>
struct BatchCfg;
template <>
struct BatchCfg<kBoxes> {
  static constexpr int NT = kThreadsBoxes, MINB = kBlocksBoxes;
};
template <>
struct BatchCfg<kGather> {
  // four resident CTAs like the single-domain gather kernel: measured faster
  // on 256 instances (24.4 vs 21.2 GLUPS with claimed items) than three,
  // although the item loop and form dispatch then spill a few registers
  static constexpr int NT = kThreadsGather, MINB = kBlocksGather;
};

// `tickets` counts the items claimed in this launch (zero at its start).
template <class ST, int MODE, int TY>
__global__ void __launch_bounds__(BatchCfg<MODE>::NT, BatchCfg<MODE>::MINB)
    k_step_batch(const StepArgs* __restrict__ table, const int4* __restrict__ items, int nitems,
                 int bp, unsigned* __restrict__ tickets) {
  constexpr int NT = BatchCfg<MODE>::NT;
  constexpr bool kAsync = sizeof(typename ST::T) == 4;
  extern __shared__ __align__(128) unsigned char sm[];
  // the arguments of this item and of the next one (two buffers)
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * kArgsBytes);
  // the item indices of the two buffers (slot p: the item whose arguments
  // buffer p receives next)
  int* slot = reinterpret_cast<int*>(sm + 2 * kArgsBytes + 8);
  // the descriptors of this item and of the next one (two slots)
  int4* desc = reinterpret_cast<int4*>(sm + 2 * kArgsBytes + 16);
  unsigned char* bx = sm + 2 * kArgsBytes + 128;
  unsigned char* fs = bx + (MODE == kBoxes ? Boxes<ST>::BYTES : 0);
  // Copy the arguments of item it into buffer buf by cp.async (completed by
  // the wait before the next CTA barrier).  Gathers read no tensor map, so
  // their copy starts past the three maps.
  constexpr int kFrom = MODE == kBoxes ? 0 : (int)(offsetof(StepArgs, use_tma) / 16);
  static_assert(sizeof(StepArgs) % 16 == 0, "whole 16-byte chunks");
  const auto copy_args = [&](int it, int buf) {
    if (it < nitems) {
      const int4* s = reinterpret_cast<const int4*>(&table[2 * items[it].x + bp]);
      int4* d = reinterpret_cast<int4*>(sm + buf * kArgsBytes);
      for (int w = kFrom + threadIdx.x; w < (int)(sizeof(StepArgs) / 16); w += NT)
        cp_async16(d + w, s + w, true);
      if (threadIdx.x == NT - 1) cp_async16(desc + buf, items + it, true);
    }
    cp_async_commit();
  };

  if constexpr (MODE == kBoxes) {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
    }
  }
  uint32_t parity = 0u;
  // claim a ticket: the index of an unclaimed item (>= nitems: none left)
  const auto claim = [&]() { return (int)min(atomicAdd(tickets, 1u), (unsigned)nitems); };
  // the same, stored straight into a shared-memory slot (one asm block, so
  // that no register holds the ticket across the item's passes)
  const auto claim_into = [&](int* dst) {
    asm volatile(
        "{\n .reg .u32 t;\n atom.global.add.u32 t, [%0], 1;\n min.u32 t, t, %2;\n"
        " st.shared.u32 [%1], t;\n}" ::"l"(tickets),
        "r"(smem_addr(dst)), "r"((unsigned)nitems)
        : "memory");
  };
  if (threadIdx.x == 0) slot[0] = claim();
  __syncthreads();
  int it = slot[0];
  copy_args(it, 0);
  // the item after it, published by the barrier at the top of the loop
  if (threadIdx.x == 0) slot[1] = claim();
  int buf = 0;
  while (it < nitems) {
    // this item's arguments and descriptor are in place, the next item's
    // index is in slot[buf ^ 1], and every thread is done with the other
    // buffer and slot (the previous item's): fill them with the next item's
    cp_async_wait_all();
    __syncthreads();
    const int next = slot[buf ^ 1];
    // the item after `next`, claimed now so that the atomic's round trip
    // overlaps the other warps' start of this item; slot[buf] was last read
    // before the barrier above (as this item's index), and the barrier at the
    // top of the next iteration publishes it
    if (threadIdx.x == 0) {
      if (next < nitems) claim_into(&slot[buf]);
      else slot[buf] = nitems;
    }
    const int4 item = desc[buf];
    const StepArgs& ga = table[2 * item.x + bp];
    copy_args(next, buf ^ 1);
    const StepArgs& a = *reinterpret_cast<const StepArgs*>(sm + buf * kArgsBytes);
    const int x0 = item.y, y0 = item.z;
    if constexpr (MODE == kBoxes) {
      if (tma_tile<ST>(a, x0, y0)) {
        // the tensor maps are read from the global table entry
        if (threadIdx.x == 0) issue_tma<ST>(ga, bx, bar, x0, y0);
        if (!wait_boxes(a, bar, parity)) return;
        parity ^= 1u;
      } else {
        fill_boxes<ST, NT, kAsync>(a, bx, x0, y0);
        if constexpr (kAsync) cp_async_wait_all();
        __syncthreads();
      }
    }
    run_item<ST, MODE, NT, TY>(a, ga, item.w, bx, fs, x0, y0);
    it = next;
    buf ^= 1;
  }
}

template <int MODE>
constexpr int batch_smem() {
  return 2 * kArgsBytes + 128 + (MODE == kBoxes ? Boxes<StoreF32>::BYTES : 0) + kFieldsMax;
}

template <int MODE, int TY>
cudaError_t launch_batch_mode(const StepArgs* table, const int4* items, int nitems, int bp,
                              int grid, unsigned* tickets, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_step_batch<StoreF32, MODE, TY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         batch_smem<MODE>());
    if (e != cudaSuccess) return e;
    configured = true;
  }
  // the launch claims its items from a zeroed counter
  cudaError_t e = cudaMemsetAsync(tickets, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  k_step_batch<StoreF32, MODE, TY><<<grid, BatchCfg<MODE>::NT, batch_smem<MODE>(), s>>>(
      table, items, nitems, bp, tickets);
  return cudaGetLastError();
}

}  // namespace

int batch_blocks_per_sm(int mode) {
  return mode == kBoxes ? BatchCfg<kBoxes>::MINB : BatchCfg<kGather>::MINB;
}

cudaError_t launch_batch(int mode, int rows, const StepArgs* table, const int4* items,
                         int nitems, int bp, int grid, unsigned* tickets, cudaStream_t s) {
  if (mode == kBoxes) {
    if (rows != kTY) return cudaErrorInvalidValue;
    return launch_batch_mode<kBoxes, kTY>(table, items, nitems, bp, grid, tickets, s);
  }
  if (rows == kShortRows)
    return launch_batch_mode<kGather, kShortRows>(table, items, nitems, bp, grid, tickets, s);
  if (rows != kTY) return cudaErrorInvalidValue;
  return launch_batch_mode<kGather, kTY>(table, items, nitems, bp, grid, tickets, s);
}

}  // namespace pflbm

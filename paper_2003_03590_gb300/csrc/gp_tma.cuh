// gp_tma.cuh -- persistent, TMA-pipelined float32 sweeps.
//
// Each CTA walks a list of tiles (a tile = B pencils of one axis).  Tiles move between
// HBM and a ring of S shared-memory stages with tensor-memory-accelerator bulk copies
// (cp.async.bulk.tensor, completion on an mbarrier for loads, bulk groups for stores),
// so loads of later tiles and stores of earlier ones overlap the FFT arithmetic of the
// current tile.  The arithmetic is the register Stockham engine of gp_fft.cuh with the
// pointwise flows of gp_sweep.cuh; only the data movement differs from k_sweep_*.
//
// Every wait on an mbarrier is bounded: if a copy does not complete within the bound the
// CTA records the failure in a device status word and returns after waiting (again
// bounded) for its own outstanding copies.
#pragma once
#include <cuda.h>

#include "gp_sweep.cuh"

namespace gp {

struct TmaSweepArgs {
  CUtensorMap map[GP_MAXB];   // one 3D map per field ([z][y][x], 8-byte elements)
  int count;                  // fields
  const tw_t<float>* tw_fwd;
  const tw_t<float>* tw_inv;
  const float4* ekx;
  const float4* ek2;
  float nl_coef, nl_shift;
  int op, axis, scale_inv;
  int* status;                // set to 1 when a bounded wait gives up
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false if the phase did not complete within the iteration limit
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (int i = 0; i < (1 << 22); ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(map),
               "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}
// The same copies with an L2 eviction-priority hint (a cache policy from createpolicy)
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void tma_load_3d_hint(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                                 uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, %3, "
      "%4}], [%5], %6;" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void tma_store_3d_hint(const CUtensorMap* map, const void* src, int c0, int c1, int c2,
                                                  uint64_t pol) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%2, %3, %4}], [%1], %5;" ::"l"(
                   map),
               "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// AND of a predicate over this thread's group of NB consecutive threads (its named barrier, as bsync)
template <int NB> __device__ __forceinline__ bool bar_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(group_bar<NB>()), "n"(NB)
      : "memory");
  return r != 0;
}

// tile geometry of the strided (y, z) sweeps: B pencils of length L, boxes of at most 256 along the pencil.
// L <= 256 ("swizzled" tiles): the B = 16 pencils of a tile are 128-byte rows of the box; TMA
// stores them with the 128-byte swizzle (16-byte chunk c of row r lands at chunk c ^ (r mod 8)),
// which lets a thread walk one pencil (a column of the tile) with 2-way instead of 16-way bank
// conflicts; each pencil then belongs to one warp and its exchanges use a private padded region.
#ifndef GP_TMA_SWIZZLE
#define GP_TMA_SWIZZLE 0   // measured slower on GB300 than the [pos][pencil] layout with block-wide exchanges
#endif
// z pencils at L = 512: consecutive z-elements of a pencil lie 2 MiB apart, one per z-plane, so a
// tile's box touches every plane's memory pages; the time of such a sweep follows the number of
// rows (box rows of B x-columns) more than their bytes, so z tiles are twice as wide there: 16
// pencils (128-byte rows) instead of 8 (measured at 512^3, one forward transform: 380 us against
// 646 us, where a y sweep with 8-pencil tiles takes 334 us).
template <int L> __host__ __device__ constexpr bool z_wide() { return L == 512; }
template <int L, int NSTAGE = 3, bool ZW = false> struct TmaStrided {
  static constexpr bool SWZ = GP_TMA_SWIZZLE && L <= 256;
  static constexpr int B = L >= 512 ? (ZW ? 16 : 8) : 16;
  static constexpr int TP = L / Plan<L>::E;
  static constexpr int NT = B * TP;
  static constexpr int TILE = B * L;                       // elements
  static constexpr int EXCH = SWZ ? B * contig_pitch<L>() : TILE;
  static constexpr int STAGE = ((((TILE > EXCH ? TILE : EXCH) * 8) + 1023) / 1024) * 128;   // elements, 1 KB multiple
  static constexpr int BOX = L > 256 ? 256 : L;            // pencil extent of one box
  static constexpr int NBOX = L / BOX;
  // stages: 3 (a load two tiles ahead), or 2 (one tile ahead, less shared memory: one more
  // CTA per SM)
  static constexpr int S = NSTAGE;
  static constexpr bool TWS = L <= 256;                    // twiddles in shared memory
  static constexpr int TWF = tw_size<L, false>(), TWI = tw_size<L, true>();
  static constexpr size_t TWB = TWS ? (size_t)(TWF + TWI) * 16 : 0;
  static constexpr size_t SMEM = (size_t)S * STAGE * 8 + 64 + TWB + 1024;   // + alignment slack
};
// element index of tile element i after the 128-byte swizzle (byte bits 7..9 XOR into bits 4..6)
__device__ __forceinline__ int swz128(int i) { return i ^ (((i >> 4) & 7) << 1); }
// x rows: B rows of length L; boxes of at most 256 along x; stage sized for the padded exchange layout
template <int L> struct TmaContig {
  static constexpr int TP = L / Plan<L>::E;
  // rows per tile: up to 256 threads, and a stage of at most ~36 KB so that three stages leave
  // room for two CTAs per SM
  static constexpr int BT = (256 / TP) < 1 ? 1 : ((256 / TP) > 16 ? 16 : 256 / TP);
  static constexpr int BS = 36864 / (contig_pitch<L>() * 8) < 1 ? 1 : 36864 / (contig_pitch<L>() * 8);
  static constexpr int B = BT <= BS ? BT : (BS >= 8 ? 8 : (BS >= 4 ? 4 : (BS >= 2 ? 2 : 1)));
  static constexpr int NT = B * TP;
  static constexpr int TILE = B * L;
  static constexpr int STAGE = B * contig_pitch<L>();     // elements, >= TILE
  static constexpr int BOX = L > 256 ? 256 : L;
  static constexpr int NBOX = L / BOX;
  static constexpr int S = 3;
  static constexpr bool TWS = L <= 256;
  static constexpr int TWF = tw_size<L, false>(), TWI = tw_size<L, true>();
  static constexpr size_t TWB = TWS ? (size_t)(TWF + TWI) * 16 : 0;
  static constexpr size_t SMEM = (size_t)S * STAGE * 8 + 64 + TWB;
};

// y or z pencils; tile index -> (field, x0, c), c the other coordinate (z for y pencils, y for z)
template <int L, int NSTAGE, int OP, bool ZW = false>
__global__ void __launch_bounds__(TmaStrided<L, NSTAGE, ZW>::NT) k_tma_strided(const __grid_constant__ TmaSweepArgs a) {
  using G = TmaStrided<L, NSTAGE, ZW>;
  using V = float2;
  constexpr int B = G::B, S = G::S, TILE = G::TILE, STAGE = G::STAGE, TP = G::TP;
  extern __shared__ __align__(128) unsigned char smraw[];
  // stages start on a 1 KB boundary of the shared window (the swizzle pattern is absolute)
  const uint32_t base = smem_u32(smraw);
  V* buf = reinterpret_cast<V*>(smraw + (((base + 1023u) & ~1023u) - base));
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf + (size_t)S * STAGE);
  const int tid = threadIdx.x;
  const int p = G::SWZ ? tid / TP : tid % B, t = G::SWZ ? tid % TP : tid / B;
  const int per_field = (L / B) * L;
  const int total = per_field * a.count;
  const unsigned bytes = (unsigned)TILE * 8u;

  auto coords = [&](int tile, int& f, int& x0, int& c) {
    f = tile / per_field;
    const int r = tile - f * per_field;
    x0 = (r % (L / B)) * B;
    c = r / (L / B);
  };
  auto issue_load = [&](int tile, int s) {
    int f, x0, c;
    coords(tile, f, x0, c);
    mbar_expect_tx(&bar[s], bytes);
#pragma unroll
    for (int k = 0; k < G::NBOX; ++k) {
      V* dst = buf + (size_t)s * STAGE + (size_t)k * G::BOX * B;
      if (a.axis == 1) tma_load_3d(dst, &a.map[f], &bar[s], x0, k * G::BOX, c);
      else tma_load_3d(dst, &a.map[f], &bar[s], x0, c, k * G::BOX);
    }
  };
  auto issue_store = [&](int tile, int s) {
    int f, x0, c;
    coords(tile, f, x0, c);
#pragma unroll
    for (int k = 0; k < G::NBOX; ++k) {
      const V* src = buf + (size_t)s * STAGE + (size_t)k * G::BOX * B;
      if (a.axis == 1) tma_store_3d(&a.map[f], src, x0, k * G::BOX, c);
      else tma_store_3d(&a.map[f], src, x0, c, k * G::BOX);
    }
  };

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
    for (int s = 0; s < S; ++s) {
      const int tile = blockIdx.x + s * gridDim.x;
      if (tile < total) issue_load(tile, s);
    }
  }
  float4* tws = reinterpret_cast<float4*>(bar + 8);   // 64 bytes of barriers, then the twiddles
  if constexpr (G::TWS) {
    for (int i = tid; i < G::TWF; i += blockDim.x) tws[i] = a.tw_fwd[i];
    for (int i = tid; i < G::TWI; i += blockDim.x) tws[G::TWF + i] = a.tw_inv[i];
  }
  __syncthreads();

  SweepArgs<float> sa{};
  sa.tw_fwd = G::TWS ? tws : a.tw_fwd;
  sa.tw_inv = G::TWS ? tws + G::TWF : a.tw_inv;
  sa.ekx = a.ekx;
  sa.ek2 = a.ek2;
  sa.nl_coef = a.nl_coef;
  sa.nl_shift = a.nl_shift;
  sa.op = a.op;
  sa.axis = a.axis;
  sa.scale_inv = a.scale_inv;
  bool failed = false;
  int it = 0;
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++it) {
    const int s = it % S;
    const bool ok = mbar_wait_bounded(&bar[s], (unsigned)(it / S) & 1u);
    if (!__syncthreads_and(ok)) {   // every thread takes the same decision
      failed = true;
      break;
    }
    V* sm = buf + (size_t)s * STAGE;
    int f, x0, c;
    coords(tile, f, x0, c);
    if constexpr (G::SWZ) {
      auto addr = [&](int pos) { return sm + swz128(pos * B + p); };
      LayContig<L> lay;
      sweep_op_body<OP, float, L, B, LayContig<L>, decltype(addr), true, true, G::TWS>(sa, t, p, sm, lay, addr, x0 + p,
                                                                                      c);
    } else {
      auto addr = [&](int pos) { return sm + pos * B + p; };
      LayStrided lay{B};
      sweep_op_body<OP, float, L, B, LayStrided, decltype(addr), true, false, G::TWS>(sa, t, p, sm, lay, addr, x0 + p,
                                                                                     c);
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      issue_store(tile, s);
      bulk_commit();
      if constexpr (S == 2) {
        const int nxt = tile + S * gridDim.x;   // this stage's next tile, once its store has left smem
        if (nxt < total) {
          bulk_wait_read0();
          issue_load(nxt, s);
        }
      } else if (it >= 1) {
        const int nxt = tile - gridDim.x + S * gridDim.x;   // the tile the previous stage serves next
        if (nxt < total) {
          bulk_wait_read1();                                // the previous stage's store has left smem
          issue_load(nxt, (it - 1) % S);
        }
      }
    }
  }
  if (failed) {
    if (tid == 0) atomicExch(a.status, 1);
  }
  if (tid == 0) bulk_wait_all();
  if (failed && tid == 0) {
    // let the loads still in flight land before the CTA's shared memory goes away
    for (int s = 0; s < S; ++s) mbar_wait_bounded(&bar[s], 0u), mbar_wait_bounded(&bar[s], 1u);
  }
}

// The same sweep with NG compute groups per CTA: group g takes the CTA's items g, g + NG, ...
// (item i = tile blockIdx.x + i gridDim.x, in stage i mod S), synchronises only its own threads
// (named barrier 1 + g), and its first thread stores the group's result and, once the store has
// read the stage, loads item i + S into it.  More warps compute per SM than one tile at a time
// allows when a tile's stage is large (512-point pencils: 8 warps per SM with one group).  Item
// i + S is loaded once item i is stored, by whichever group computed item i: a group waits only
// for items of lower index, so the groups cannot wait on one another in a cycle.
//
// A group may reach item i while its stage still serves item i - S of another group, whose load
// may not even have landed.  An mbarrier wait on the parity of item i's phase alone cannot tell
// that phase from the one two loads earlier (same parity, complete), so every stage also counts
// in shared memory the loads issued into it: the group first waits until the load of item i has
// been issued (its (i / S)-th load), and only then for that phase's parity.  Once that load is
// issued, the stage's barrier is in item i's phase or has just completed it: the next load into
// the stage waits for this group to finish item i.
__device__ __forceinline__ bool stage_wait(uint64_t* bar, volatile int* issued, int it, int S) {
  const int k = it / S;
  bool ok = false;
  for (int i = 0; i < (1 << 22); ++i)
    if (*issued > k) {
      ok = true;
      break;
    }
  return ok && mbar_wait_bounded(bar, (unsigned)k & 1u);
}
__device__ __forceinline__ void count_issued(volatile int* issued) {
  __threadfence_block();   // the load's arming of the barrier before the count that releases its waiters
  atomicAdd((int*)issued, 1);
}
template <int L, int NSTAGE, int OP, bool ZW, int NG>
__global__ void __launch_bounds__(NG * TmaStrided<L, NSTAGE, ZW>::NT)
    k_tma_strided_g(const __grid_constant__ TmaSweepArgs a) {
  using G = TmaStrided<L, NSTAGE, ZW>;
  using V = float2;
  static_assert(!G::SWZ, "grouped sweeps use the [pos][pencil] tile layout");
  constexpr int B = G::B, S = G::S, TILE = G::TILE, STAGE = G::STAGE, NTG = G::NT;
  extern __shared__ __align__(128) unsigned char smraw[];
  const uint32_t base = smem_u32(smraw);
  V* buf = reinterpret_cast<V*>(smraw + (((base + 1023u) & ~1023u) - base));
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf + (size_t)S * STAGE);
  const int tid = threadIdx.x, grp = tid / NTG, lt = tid % NTG;
  const int p = lt % B, t = lt / B;
  const bool leader = lt == 0;
  const int per_field = (L / B) * L;
  const int total = per_field * a.count;
  const unsigned bytes = (unsigned)TILE * 8u;
  auto coords = [&](int tile, int& f, int& x0, int& c) {
    f = tile / per_field;
    const int r = tile - f * per_field;
    x0 = (r % (L / B)) * B;
    c = r / (L / B);
  };
  auto issue_load = [&](int tile, int s) {
    int f, x0, c;
    coords(tile, f, x0, c);
    mbar_expect_tx(&bar[s], bytes);
#pragma unroll
    for (int k = 0; k < G::NBOX; ++k) {
      V* dst = buf + (size_t)s * STAGE + (size_t)k * G::BOX * B;
      if (a.axis == 1) tma_load_3d(dst, &a.map[f], &bar[s], x0, k * G::BOX, c);
      else tma_load_3d(dst, &a.map[f], &bar[s], x0, c, k * G::BOX);
    }
  };
  auto issue_store = [&](int tile, int s) {
    int f, x0, c;
    coords(tile, f, x0, c);
#pragma unroll
    for (int k = 0; k < G::NBOX; ++k) {
      const V* src = buf + (size_t)s * STAGE + (size_t)k * G::BOX * B;
      if (a.axis == 1) tma_store_3d(&a.map[f], src, x0, k * G::BOX, c);
      else tma_store_3d(&a.map[f], src, x0, c, k * G::BOX);
    }
  };
  volatile int* issued = reinterpret_cast<volatile int*>(bar + 4);   // loads issued per stage
  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
    for (int s = 0; s < S; ++s) {
      const int tile = blockIdx.x + s * gridDim.x;
      issued[s] = 0;
      if (tile < total) {
        issue_load(tile, s);
        issued[s] = 1;
      }
    }
  }
  float4* tws = reinterpret_cast<float4*>(bar + 8);
  if constexpr (G::TWS) {
    for (int i = tid; i < G::TWF; i += blockDim.x) tws[i] = a.tw_fwd[i];
    for (int i = tid; i < G::TWI; i += blockDim.x) tws[G::TWF + i] = a.tw_inv[i];
  }
  __syncthreads();
  SweepArgs<float> sa{};
  sa.tw_fwd = G::TWS ? tws : a.tw_fwd;
  sa.tw_inv = G::TWS ? tws + G::TWF : a.tw_inv;
  sa.ekx = a.ekx;
  sa.ek2 = a.ek2;
  sa.nl_coef = a.nl_coef;
  sa.nl_shift = a.nl_shift;
  sa.op = a.op;
  sa.axis = a.axis;
  sa.scale_inv = a.scale_inv;
  bool failed = false;
  for (int it = grp;; it += NG) {
    const int tile = blockIdx.x + it * gridDim.x;
    if (tile >= total) break;
    const int s = it % S;
    if (!bar_and<NTG>(stage_wait(&bar[s], issued + s, it, S))) {   // every thread of the group takes the same decision
      failed = true;
      break;
    }
    V* sm = buf + (size_t)s * STAGE;
    int f, x0, c;
    coords(tile, f, x0, c);
    auto addr = [&](int pos) { return sm + pos * B + p; };
    LayStrided lay{B};
    sweep_op_body<OP, float, L, B, LayStrided, decltype(addr), true, false, G::TWS, NTG>(sa, t, p, sm, lay, addr,
                                                                                       x0 + p, c);
    fence_async_smem();
    bsync<NTG>();
    if (leader) {
      issue_store(tile, s);
      bulk_commit();
      const int nxt = tile + S * gridDim.x;   // item it + S, in this stage once the store has read it
      if (nxt < total) {
        bulk_wait_read0();
        issue_load(nxt, s);
        count_issued(issued + s);
      }
    }
  }
  if (failed && leader) atomicExch(a.status, 1);
  if (leader) bulk_wait_all();
  if (__syncthreads_or(failed) && tid == 0) {
    // let the loads still in flight land before the CTA's shared memory goes away
    for (int s = 0; s < S; ++s) mbar_wait_bounded(&bar[s], 0u), mbar_wait_bounded(&bar[s], 1u);
  }
}

// x rows; tile index -> (field, row0); row = y + N z
template <int L, int OP>
__global__ void __launch_bounds__(TmaContig<L>::NT) k_tma_contig(const __grid_constant__ TmaSweepArgs a) {
  using G = TmaContig<L>;
  using V = float2;
  constexpr int B = G::B, S = G::S, TILE = G::TILE, STAGE = G::STAGE, TP = G::TP;
  extern __shared__ __align__(128) unsigned char smraw[];
  V* buf = reinterpret_cast<V*>(smraw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + (size_t)S * STAGE * 8);
  const int tid = threadIdx.x, p = tid / TP, t = tid % TP;
  const int per_field = L * L / B;
  const int total = per_field * a.count;
  const unsigned bytes = (unsigned)TILE * 8u;

  auto issue_load = [&](int tile, int s) {
    const int f = tile / per_field, row0 = (tile - f * per_field) * B;
    mbar_expect_tx(&bar[s], bytes);
#pragma unroll
    for (int k = 0; k < G::NBOX; ++k)
      tma_load_3d(buf + (size_t)s * STAGE + (size_t)k * G::BOX * B, &a.map[f], &bar[s], k * G::BOX, row0 % L, row0 / L);
  };
  auto issue_store = [&](int tile, int s) {
    const int f = tile / per_field, row0 = (tile - f * per_field) * B;
#pragma unroll
    for (int k = 0; k < G::NBOX; ++k)
      tma_store_3d(&a.map[f], buf + (size_t)s * STAGE + (size_t)k * G::BOX * B, k * G::BOX, row0 % L, row0 / L);
  };

  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
    for (int s = 0; s < S; ++s) {
      const int tile = blockIdx.x + s * gridDim.x;
      if (tile < total) issue_load(tile, s);
    }
  }
  float4* tws = reinterpret_cast<float4*>(bar + 8);   // 64 bytes of barriers, then the twiddles
  if constexpr (G::TWS) {
    for (int i = tid; i < G::TWF; i += blockDim.x) tws[i] = a.tw_fwd[i];
    for (int i = tid; i < G::TWI; i += blockDim.x) tws[G::TWF + i] = a.tw_inv[i];
  }
  __syncthreads();

  SweepArgs<float> sa{};
  sa.tw_fwd = G::TWS ? tws : a.tw_fwd;
  sa.tw_inv = G::TWS ? tws + G::TWF : a.tw_inv;
  sa.ekx = a.ekx;
  sa.ek2 = a.ek2;
  sa.nl_coef = a.nl_coef;
  sa.nl_shift = a.nl_shift;
  sa.op = a.op;
  sa.axis = a.axis;
  sa.scale_inv = a.scale_inv;
  LayContig<L> lay;
  bool failed = false;
  int it = 0;
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x, ++it) {
    const int s = it % S;
    const bool ok = mbar_wait_bounded(&bar[s], (unsigned)(it / S) & 1u);
    if (!__syncthreads_and(ok)) {
      failed = true;
      break;
    }
    V* sm = buf + (size_t)s * STAGE;
    const int f = tile / per_field, row = (tile - f * per_field) * B + p;
    // the TMA tile is [box k][row][x within box]
    auto addr = [&](int pos) { return sm + (pos / G::BOX) * (G::BOX * B) + p * G::BOX + (pos % G::BOX); };
    sweep_op_body<OP, float, L, B, LayContig<L>, decltype(addr), true, (TP <= 32), G::TWS>(sa, t, p, sm, lay, addr, row % L,
                                                                                       row / L);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      issue_store(tile, s);
      bulk_commit();
      if (it >= 1) {
        const int nxt = tile - gridDim.x + S * gridDim.x;
        if (nxt < total) {
          bulk_wait_read1();
          issue_load(nxt, (it - 1) % S);
        }
      }
    }
  }
  if (failed) {
    if (tid == 0) atomicExch(a.status, 1);
  }
  if (tid == 0) bulk_wait_all();
  if (failed && tid == 0) {
    for (int s = 0; s < S; ++s) mbar_wait_bounded(&bar[s], 0u), mbar_wait_bounded(&bar[s], 1u);
  }
}

// x rows with NG compute groups per CTA (as k_tma_strided_g)
template <int L, int OP, int NG>
__global__ void __launch_bounds__(NG * TmaContig<L>::NT, 2) k_tma_contig_g(const __grid_constant__ TmaSweepArgs a) {
  using G = TmaContig<L>;
  using V = float2;
  constexpr int B = G::B, S = G::S, TILE = G::TILE, STAGE = G::STAGE, TP = G::TP, NTG = G::NT;
  extern __shared__ __align__(128) unsigned char smraw[];
  V* buf = reinterpret_cast<V*>(smraw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + (size_t)S * STAGE * 8);
  const int tid = threadIdx.x, grp = tid / NTG, lt = tid % NTG;
  const int p = lt / TP, t = lt % TP;
  const bool leader = lt == 0;
  const int per_field = L * L / B;
  const int total = per_field * a.count;
  const unsigned bytes = (unsigned)TILE * 8u;
  auto issue_load = [&](int tile, int s) {
    const int f = tile / per_field, row0 = (tile - f * per_field) * B;
    mbar_expect_tx(&bar[s], bytes);
#pragma unroll
    for (int k = 0; k < G::NBOX; ++k)
      tma_load_3d(buf + (size_t)s * STAGE + (size_t)k * G::BOX * B, &a.map[f], &bar[s], k * G::BOX, row0 % L, row0 / L);
  };
  auto issue_store = [&](int tile, int s) {
    const int f = tile / per_field, row0 = (tile - f * per_field) * B;
#pragma unroll
    for (int k = 0; k < G::NBOX; ++k)
      tma_store_3d(&a.map[f], buf + (size_t)s * STAGE + (size_t)k * G::BOX * B, k * G::BOX, row0 % L, row0 / L);
  };
  volatile int* issued = reinterpret_cast<volatile int*>(bar + 4);   // loads issued per stage
  if (tid == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
    for (int s = 0; s < S; ++s) {
      const int tile = blockIdx.x + s * gridDim.x;
      issued[s] = 0;
      if (tile < total) {
        issue_load(tile, s);
        issued[s] = 1;
      }
    }
  }
  float4* tws = reinterpret_cast<float4*>(bar + 8);
  if constexpr (G::TWS) {
    for (int i = tid; i < G::TWF; i += blockDim.x) tws[i] = a.tw_fwd[i];
    for (int i = tid; i < G::TWI; i += blockDim.x) tws[G::TWF + i] = a.tw_inv[i];
  }
  __syncthreads();
  SweepArgs<float> sa{};
  sa.tw_fwd = G::TWS ? tws : a.tw_fwd;
  sa.tw_inv = G::TWS ? tws + G::TWF : a.tw_inv;
  sa.ekx = a.ekx;
  sa.ek2 = a.ek2;
  sa.nl_coef = a.nl_coef;
  sa.nl_shift = a.nl_shift;
  sa.op = a.op;
  sa.axis = a.axis;
  sa.scale_inv = a.scale_inv;
  LayContig<L> lay;
  bool failed = false;
  for (int it = grp;; it += NG) {
    const int tile = blockIdx.x + it * gridDim.x;
    if (tile >= total) break;
    const int s = it % S;
    if (!bar_and<NTG>(stage_wait(&bar[s], issued + s, it, S))) {
      failed = true;
      break;
    }
    V* sm = buf + (size_t)s * STAGE;
    const int f = tile / per_field, row = (tile - f * per_field) * B + p;
    auto addr = [&](int pos) { return sm + (pos / G::BOX) * (G::BOX * B) + p * G::BOX + (pos % G::BOX); };
    sweep_op_body<OP, float, L, B, LayContig<L>, decltype(addr), true, (TP <= 32), G::TWS, NTG>(sa, t, p, sm, lay, addr,
                                                                                              row % L, row / L);
    fence_async_smem();
    bsync<NTG>();
    if (leader) {
      issue_store(tile, s);
      bulk_commit();
      const int nxt = tile + S * gridDim.x;
      if (nxt < total) {
        bulk_wait_read0();
        issue_load(nxt, s);
        count_issued(issued + s);
      }
    }
  }
  if (failed && leader) atomicExch(a.status, 1);
  if (leader) bulk_wait_all();
  if (__syncthreads_or(failed) && tid == 0) {
    for (int s = 0; s < S; ++s) mbar_wait_bounded(&bar[s], 0u), mbar_wait_bounded(&bar[s], 1u);
  }
}

// Launchers: one kernel per (stages, operation); the grid is the CTAs that fit per SM (or
// ctas_per_sm if smaller) times the SMs, at most one CTA per tile.
// grouped kernels (two compute groups per CTA) exist for the lengths whose stages are large
template <int L> __host__ __device__ constexpr bool grouped_ok() { return L >= 512; }

template <int L> struct TmaLaunch {
  template <class Kern> static int occupancy(Kern k, int threads, size_t smem) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem);
    return nb;
  }
  static int sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
  }
  // CTAs per SM of every (kernel, operation), queried together on the first launch of this
  // length (which is never inside a stream capture: a step's first sweeps run directly)
  enum { K_S2 = 0, K_S3 = 8, K_C = 16, K_Z2 = 24, K_Z3 = 32, K_GS = 40, K_GZ = 48, K_GC = 56 };
  static constexpr bool ZWS = z_wide<L>();
  static const int* occ_table() {
    static int t[64] = {};
    static bool done = false;
    if (!done) {
#define GP_OCC_S(OPV)                                                                                       \
  t[K_S2 + OPV] = occupancy(k_tma_strided<L, 2, OPV>, TmaStrided<L, 2>::NT, TmaStrided<L, 2>::SMEM);           \
  t[K_S3 + OPV] = occupancy(k_tma_strided<L, 3, OPV>, TmaStrided<L, 3>::NT, TmaStrided<L, 3>::SMEM);
#define GP_OCC_Z(OPV)                                                                                                   \
  t[K_Z2 + OPV] = occupancy(k_tma_strided<L, 2, OPV, true>, TmaStrided<L, 2, true>::NT, TmaStrided<L, 2, true>::SMEM); \
  t[K_Z3 + OPV] = occupancy(k_tma_strided<L, 3, OPV, true>, TmaStrided<L, 3, true>::NT, TmaStrided<L, 3, true>::SMEM);
#define GP_OCC_C(OPV) t[K_C + OPV] = occupancy(k_tma_contig<L, OPV>, TmaContig<L>::NT, TmaContig<L>::SMEM);
#define GP_OCC_G(OPV)                                                                                                 \
  t[K_GS + OPV] = occupancy(k_tma_strided_g<L, 3, OPV, false, 2>, 2 * TmaStrided<L, 3>::NT, TmaStrided<L, 3>::SMEM);   \
  t[K_GZ + OPV] = occupancy(k_tma_strided_g<L, 3, OPV, ZWS, 2>, 2 * TmaStrided<L, 3, ZWS>::NT, TmaStrided<L, 3, ZWS>::SMEM);
#define GP_OCC_GC(OPV) t[K_GC + OPV] = occupancy(k_tma_contig_g<L, OPV, 2>, 2 * TmaContig<L>::NT, TmaContig<L>::SMEM);
      GP_STRIDED_OPS(GP_OCC_S)
      if constexpr (z_wide<L>()) { GP_STRIDED_OPS(GP_OCC_Z) }
      GP_CONTIG_OPS(GP_OCC_C)
      if constexpr (grouped_ok<L>()) {
        GP_STRIDED_OPS(GP_OCC_G)
        GP_CONTIG_OPS(GP_OCC_GC)
      }
#undef GP_OCC_S
#undef GP_OCC_Z
#undef GP_OCC_C
#undef GP_OCC_G
#undef GP_OCC_GC
      done = true;
    }
    return t;
  }
  static int grid_of(int occ, int ctas_per_sm, int tiles) {
    const int grid = sms() * (ctas_per_sm > 0 && ctas_per_sm < occ ? ctas_per_sm : occ);
    return grid > tiles ? tiles : grid;
  }
  template <int NSTAGE, int OP, bool ZW = false>
  static cudaError_t strided(const TmaSweepArgs& a, int ctas_per_sm, cudaStream_t s) {
    using G = TmaStrided<L, NSTAGE, ZW>;
    const int occ = occ_table()[(ZW ? (NSTAGE == 2 ? K_Z2 : K_Z3) : (NSTAGE == 2 ? K_S2 : K_S3)) + OP];
    if (occ < 1) return cudaErrorInvalidConfiguration;
    k_tma_strided<L, NSTAGE, OP, ZW><<<grid_of(occ, ctas_per_sm, ((L / G::B) * L) * a.count), G::NT, G::SMEM, s>>>(a);
    return cudaGetLastError();
  }
  template <int OP, bool ZW> static cudaError_t strided_g(const TmaSweepArgs& a, int ctas_per_sm, cudaStream_t s) {
    using G = TmaStrided<L, 3, ZW>;
    const int occ = occ_table()[(ZW ? K_GZ : K_GS) + OP];
    if (occ < 1) return cudaErrorInvalidConfiguration;
    k_tma_strided_g<L, 3, OP, ZW, 2><<<grid_of(occ, ctas_per_sm, ((L / G::B) * L) * a.count), 2 * G::NT, G::SMEM, s>>>(a);
    return cudaGetLastError();
  }
  template <int OP> static cudaError_t contig(const TmaSweepArgs& a, int ctas_per_sm, cudaStream_t s) {
    using G = TmaContig<L>;
    const int occ = occ_table()[K_C + OP];
    if (occ < 1) return cudaErrorInvalidConfiguration;
    k_tma_contig<L, OP><<<grid_of(occ, ctas_per_sm, (L * L / G::B) * a.count), G::NT, G::SMEM, s>>>(a);
    return cudaGetLastError();
  }
  template <int OP> static cudaError_t contig_g(const TmaSweepArgs& a, int ctas_per_sm, cudaStream_t s) {
    using G = TmaContig<L>;
    const int occ = occ_table()[K_GC + OP];
    if (occ < 1) return cudaErrorInvalidConfiguration;
    k_tma_contig_g<L, OP, 2><<<grid_of(occ, ctas_per_sm, (L * L / G::B) * a.count), 2 * G::NT, G::SMEM, s>>>(a);
    return cudaGetLastError();
  }
  // stages: 3 or 2 (y/z sweeps only); groups: 1, or 2 compute groups per CTA (lengths >= 512,
  // three stages)
  static cudaError_t launch(const TmaSweepArgs& a, int ctas_per_sm, int stages, int groups, cudaStream_t s) {
    if constexpr (grouped_ok<L>()) {
      if (groups == 2) {
#define GP_OP_CASE_GC(OPV) \
  case OPV: return contig_g<OPV>(a, ctas_per_sm, s);
#define GP_OP_CASE_GS(OPV) \
  case OPV: return strided_g<OPV, false>(a, ctas_per_sm, s);
#define GP_OP_CASE_GZ(OPV) \
  case OPV: return strided_g<OPV, ZWS>(a, ctas_per_sm, s);
        if (a.axis == 0) {
          switch (a.op) { GP_CONTIG_OPS(GP_OP_CASE_GC) default: return cudaErrorInvalidValue; }
        }
        if (a.axis == 2) {
          switch (a.op) { GP_STRIDED_OPS(GP_OP_CASE_GZ) default: return cudaErrorInvalidValue; }
        }
        switch (a.op) { GP_STRIDED_OPS(GP_OP_CASE_GS) default: return cudaErrorInvalidValue; }
#undef GP_OP_CASE_GC
#undef GP_OP_CASE_GS
#undef GP_OP_CASE_GZ
      }
    }
    if (groups != 1) return cudaErrorInvalidValue;
#define GP_OP_CASE_C(OPV) \
  case OPV: return contig<OPV>(a, ctas_per_sm, s);
#define GP_OP_CASE_S2(OPV) \
  case OPV: return strided<2, OPV>(a, ctas_per_sm, s);
#define GP_OP_CASE_S3(OPV) \
  case OPV: return strided<3, OPV>(a, ctas_per_sm, s);
    if (a.axis == 0) {
      switch (a.op) { GP_CONTIG_OPS(GP_OP_CASE_C) default: return cudaErrorInvalidValue; }
    }
    if constexpr (z_wide<L>()) {
      if (a.axis == 2) {
#define GP_OP_CASE_Z2(OPV) \
  case OPV: return strided<2, OPV, true>(a, ctas_per_sm, s);
#define GP_OP_CASE_Z3(OPV) \
  case OPV: return strided<3, OPV, true>(a, ctas_per_sm, s);
        if (stages == 2) {
          switch (a.op) { GP_STRIDED_OPS(GP_OP_CASE_Z2) default: return cudaErrorInvalidValue; }
        }
        switch (a.op) { GP_STRIDED_OPS(GP_OP_CASE_Z3) default: return cudaErrorInvalidValue; }
#undef GP_OP_CASE_Z2
#undef GP_OP_CASE_Z3
      }
    }
    if (stages == 2) {
      switch (a.op) { GP_STRIDED_OPS(GP_OP_CASE_S2) default: return cudaErrorInvalidValue; }
    }
    switch (a.op) { GP_STRIDED_OPS(GP_OP_CASE_S3) default: return cudaErrorInvalidValue; }
#undef GP_OP_CASE_C
#undef GP_OP_CASE_S2
#undef GP_OP_CASE_S3
  }
};

}  // namespace gp

// gp_plane.cuh -- the three sweeps of a time step that stay inside one z-plane, fused into one
// persistent kernel.
//
// Of the four sweeps of a float32 step (gp_step.cu), three touch a z-plane only through
// that plane: forward y, then forward x + K(s) + inverse x, then inverse y.  One plane of
// one field is therefore an independent unit of three phases:
//   phase 0  forward y transforms of the plane's N / B column tiles (B x-columns each),
//   phase 1  forward x, K(s) with 1/N^3, inverse x of its N / B row tiles (B rows each),
//   phase 2  inverse y transforms of its column tiles,
// where phase q + 1 of a plane may start once every tile of phase q of that plane is stored.
// The kernel hands out tiles ("items") from a global ticket counter in an order where phase
// q + 1 of plane u follows phase q of plane u by a lag of D planes' worth of items: items
// that depend on one another are far apart in the order, so a CTA almost never waits, and
// the planes between the phases of one plane (2 D planes) are the only data in flight --
// a few tens of MB, which stay in the 126 MB L2: phases 1 and 2 read what phases 0 and 1
// wrote from L2, and the field crosses HBM about once in each direction.  The memory-bound
// y tiles and the arithmetic-bound x tiles also run side by side on the SMs instead of in
// separate launches.
//
// Roles.  The last warp of a CTA is a producer: one thread claims tickets (two per atomic,
// the next claim issued an item ahead), waits for each item's inputs, issues its TMA load
// into a ring of S shared-memory stages, issues the TMA store once the compute warps
// signal (an mbarrier per stage) that the stage holds the result, and counts the stored
// tile.  The compute warps only wait for loaded stages; their exchanges use a named barrier
// that leaves the producer out, so no fence or L2 round trip of the bookkeeping sits
// between two tiles of the compute warps.
//
// Synchronisation.  Completed tiles are counted per (plane, phase) in global memory.  A tile
// is counted only after its TMA store has completed (bulk wait_group), followed by a
// proxy fence and a release add; a dependent tile is loaded only after a relaxed read of the
// count has seen every tile of the phase it needs, then an acquire fence and a proxy fence
// (TMA copies are in the async proxy).  The producer never blocks: it polls, in one loop,
// for computed stages to store and for the next item's inputs, and counts its own newest
// stored tile before it waits for other CTAs' tiles -- so the oldest unfinished item of the
// launch can always proceed.  Every wait is bounded; a wait that gives up sets the status
// word (the result is then invalid, the launch still ends).
#pragma once
#include "gp_tma.cuh"

namespace gp {

struct TmaPlaneArgs {
  CUtensorMap map_y[GP_MAXB];   // per field: boxes of B x-columns by (up to 256) y
  CUtensorMap map_x[GP_MAXB];   // per field: boxes of (up to 256) x by B rows
  int count;                    // fields
  const tw_t<float>* tw_fwd;
  const tw_t<float>* tw_inv;
  const float4* ekx;            // K(s) factor along x, hi/lo pairs
  const float4* ek2;            // K(s) factor of (y, z) with 1/N^3, hi/lo pairs, index z * N + y
  int lag;                      // D: planes between consecutive phases of a plane in the order
  int* sync;                    // [0] ticket counter; [1 + 2 u + q] stored tiles of phase q of plane u
  int* status;                  // set to 1 when a bounded wait gives up
  int skip;                     // tickets never handed out (0; a test of the bounded waits sets it)
};

// NS: shared-memory stages, 3, or 2 with the twiddles read through L1 instead of shared memory
// (one more CTA per SM at 256, registers capped to fit three).  NG: compute groups per CTA (1, or
// several for the 512-point lengths, whose one group of 4 warps per tile leaves the SM short of
// warps; one CTA per SM then, with NS = NG + 2 stages).
template <int L, int NS = 3, int NG = 1> struct TmaPlane {
  static constexpr int B = TmaStrided<L>::B;               // pencils (columns or rows) per tile
  static constexpr int TP = L / Plan<L>::E;                // threads per pencil
  static constexpr int NC = B * TP;                        // compute threads of one group
  static constexpr int NT = NG * NC + 64;                  // + a loader warp and a storer warp
  static constexpr int Q = L / B;                          // tiles per phase and plane
  static constexpr int TILE = B * L;                       // elements
  static constexpr int STAGE_C = B * contig_pitch<L>();    // rows use a padded exchange layout
  static constexpr int STAGE = ((STAGE_C > TILE ? STAGE_C : TILE) + 15) / 16 * 16;   // 128-byte multiple
  static constexpr int BOX = L > 256 ? 256 : L;
  static constexpr int NBOX = L / BOX;
  static constexpr int S = NS;
  static constexpr int CHUNK = 2;                          // tickets taken per atomic
  static constexpr bool TWS = L <= 256 && NS == 3;
  // CTAs per SM the registers must allow (shared memory allows one at 1024)
  static constexpr int MINB = NG > 1 ? 1 : ((NS == 2 && L <= 256) ? 3 : (L >= 1024 ? 1 : 2));
  static constexpr int TWF = tw_size<L, false>(), TWI = tw_size<L, true>();
  static constexpr size_t TWB = TWS ? (size_t)(TWF + TWI) * 16 : 0;
  static_assert(NS <= 8, "barrier arrays hold 8 stages");
  static constexpr size_t SMEM = (size_t)S * STAGE * 8 + 192 + 64 + TWB + 128;   // barriers, ring and counts, twiddles, slack
};

__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void red_release_gpu_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait1() { asm volatile("cp.async.bulk.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait2() { asm volatile("cp.async.bulk.wait_group 2;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}


// Item order.  Blocks of Q items (one phase of one plane) are ordered by "group" g: group g
// holds phase 0 of plane g, phase 1 of plane g - D and phase 2 of plane g - 2D (those that
// exist), in that order.  C(g) = number of blocks in groups before g.
__device__ __forceinline__ int plane_blocks_before(int g, int U, int D) {
  int c = 0;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int v = g - q * D;
    c += v < 0 ? 0 : (v > U ? U : v);
  }
  return c;
}
template <int Q>
__device__ __forceinline__ void plane_item(int ticket, int U, int D, int& ph, int& u, int& j) {
  const int b = ticket / Q;
  j = ticket - b * Q;
  int lo = 0, hi = U + 2 * D;   // C(lo) <= b < C(hi)
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (plane_blocks_before(mid, U, D) <= b) lo = mid;
    else hi = mid;
  }
  int r = b - plane_blocks_before(lo, U, D);
  ph = 0;
  u = lo;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int v = lo - q * D;
    if (v >= 0 && v < U) {
      if (r == 0) {
        ph = q;
        u = v;
        return;
      }
      --r;
    }
  }
}

template <int L, int NS, int NG>
__global__ void __launch_bounds__(TmaPlane<L, NS, NG>::NT, TmaPlane<L, NS, NG>::MINB)
    k_tma_plane(const __grid_constant__ TmaPlaneArgs a) {
  using G = TmaPlane<L, NS, NG>;
  using V = float2;
  constexpr int B = G::B, S = G::S, STAGE = G::STAGE, TP = G::TP, Q = G::Q, BOX = G::BOX, NC = G::NC;
  constexpr int NCT = NG * NC;                                             // compute threads of the CTA
  extern __shared__ __align__(128) unsigned char smraw[];
  const uint32_t base = smem_u32(smraw);
  V* buf = reinterpret_cast<V*>(smraw + (((base + 127u) & ~127u) - base));
  uint64_t* full = reinterpret_cast<uint64_t*>(buf + (size_t)S * STAGE);   // data of stage s landed
  uint64_t* empty = full + 8;                                              // compute of stage s done
  uint64_t* freed = full + 16;                                             // stage s stored (read)
  int* ring = reinterpret_cast<int*>(full + 24);  // [s]: packed item of stage s, -1: no more items
  volatile int* issued = ring + 8;                // [s]: items the loader has put into stage s
  float4* tws = reinterpret_cast<float4*>(ring + 16);
  const int tid = threadIdx.x;

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NC);
      mbar_init(&freed[s], 1);
      issued[s] = 0;
    }
    fence_mbar_init();
  }
  if constexpr (G::TWS) {
    for (int i = tid; i < G::TWF; i += blockDim.x) tws[i] = a.tw_fwd[i];
    for (int i = tid; i < G::TWI; i += blockDim.x) tws[G::TWF + i] = a.tw_inv[i];
  }
  __syncthreads();

  // L2 priorities: the phase-0 loads (the plane as the z sweep left it, read once here) and the
  // phase-2 stores (the step's output) go first; the plane between its phases (stored by
  // phases 0 and 1, read back by phases 1 and 2) stays, so that it does not round-trip to HBM
  uint64_t pol_first = 0, pol_last = 0;
  if (tid >= NG * NC) {
    pol_first = l2_policy_evict_first();
    pol_last = l2_policy_evict_last();
  }
  auto copy_tile = [&](int it, int s, bool load) {   // TMA copy of item `it` between HBM/L2 and stage s
    const int ph = it & 3, j = (it >> 2) & 511, u = it >> 11;
    const int f = u / L, z = u - f * L;
    V* st = buf + (size_t)s * STAGE;
    const uint64_t pol = (load ? ph == 0 : ph == 2) ? pol_first : pol_last;
#pragma unroll
    for (int k = 0; k < G::NBOX; ++k) {
      V* sk = st + (size_t)k * BOX * B;
      if (ph == 1) {
        if (load) tma_load_3d_hint(sk, &a.map_x[f], &full[s], k * BOX, j * B, z, pol);
        else tma_store_3d_hint(&a.map_x[f], sk, k * BOX, j * B, z, pol);
      } else {
        if (load) tma_load_3d_hint(sk, &a.map_y[f], &full[s], j * B, k * BOX, z, pol);
        else tma_store_3d_hint(&a.map_y[f], sk, j * B, k * BOX, z, pol);
      }
    }
  };

  if (tid >= NCT) {
    // -------------------------------------------------------- loader (warp NCT/32) and storer (warp NCT/32 + 1)
    if ((tid - NCT) % 32 != 0) return;
    const bool loader = tid == NCT;
    const int U = a.count * L;
    const int total = 3 * U * Q;
    const int D = a.lag;
    int* const done = a.sync + 1;
    int idle = 0;
    auto stalled = [&]() -> bool {   // bounded idling: ~1 s without progress gives up
      if (++idle > (1 << 21)) return true;
      __nanosleep(32);
      return false;
    };
    if (loader) {
      constexpr int CHUNK = G::CHUNK;
      int c_next = 0, c_end = 0;     // current chunk of tickets [c_next, c_end)
      int pend = -1, pend_seen = 0;  // next item and the count last seen for it
      bool exhausted = false;
      int* acq_ctr = nullptr;        // counter already acquired complete by this thread
      auto dep_count = [&](int it) -> int {
        const int ph = it & 3;
        return ph == 0 ? Q : ld_relaxed_gpu(done + 2 * (it >> 11) + ph - 1);
      };
      auto claim = [&]() {   // make `pend` the next item in ticket order and start reading its count
        if (pend >= 0 || exhausted) return;
        if (c_next >= c_end) {
          const int t0 = atomicAdd(a.sync, CHUNK) + a.skip;
          if (t0 >= total) {
            exhausted = true;
            return;
          }
          c_next = t0;
          c_end = t0 + CHUNK < total ? t0 + CHUNK : total;
        }
        int ph, u, j;
        plane_item<Q>(c_next++, U, D, ph, u, j);
        pend = ph | (j << 2) | (u << 11);
        pend_seen = dep_count(pend);
      };
      bool gave_up = false;
      int i = 0;
      claim();
      for (; pend >= 0; ++i) {
        const int s = i % S;
        // the stage is free once the storer has stored its previous item
        idle = 0;
        while (i >= S && !mbar_try_wait(&freed[s], (unsigned)(i / S - 1) & 1u))
          if ((gave_up = stalled())) break;
        if (gave_up) break;
        idle = 0;
        while (pend_seen < Q) {
          pend_seen = dep_count(pend);
          if (pend_seen < Q && (gave_up = stalled())) break;
        }
        if (gave_up) break;
        ring[s] = pend;
        if ((pend & 3) > 0) {
          int* c = done + 2 * (pend >> 11) + (pend & 3) - 1;
          if (c != acq_ctr) {
            fence_acq_rel_gpu();    // with the relaxed read of the count: acquire the tiles it counts
            fence_async_global();   // ... for the TMA (async proxy) reads below
            acq_ctr = c;
          }
        }
        mbar_expect_tx(&full[s], (unsigned)G::TILE * 8u);
        copy_tile(pend, s, true);
        if constexpr (NG > 1) count_issued(issued + s);
        pend = -1;
        claim();   // the next item's ticket and count are read while this one loads
      }
      if (gave_up) atomicExch(a.status, 1);
      // end markers at items i .. i + NG - 1, one for each compute group (each group stops at the
      // first marker it meets); the storer stops after i items
      for (int q = 0; q < NG; ++q) {
        const int e = i + q;
        if (e >= S) {
          idle = 0;
          while (!mbar_try_wait(&freed[e % S], (unsigned)(e / S - 1) & 1u))
            if (stalled()) break;
        }
        ring[e % S] = -1;
        if constexpr (NG > 1) count_issued(issued + e % S);
        mbar_arrive(&full[e % S]);   // release: ring[] is visible to the waiters of full[]
      }
      return;
    }
    // storer: store each computed stage, free it once read, count it once complete
    int unrel = -1;   // stored item whose count is pending (its store may be in flight)
    auto count_item = [&](int it) {
      if ((it & 3) < 2) {
        fence_async_global();
        red_release_gpu_add(done + 2 * (it >> 11) + (it & 3), 1);
      }
    };
    bool gave_up = false;
    for (int k = 0;; ++k) {
      const int s = k % S;
      idle = 0;
      bool ready = false;
      while (!(ready = mbar_try_wait(&empty[s], (unsigned)(k / S) & 1u))) {
        if (unrel >= 0) {   // idle: finish and count the pending store now
          bulk_wait_all();
          count_item(unrel);
          unrel = -1;
        }
        if (mbar_try_wait(&full[s], (unsigned)(k / S) & 1u) && ring[s] < 0) break;   // end marker
        if ((gave_up = stalled())) break;
      }
      if (!ready) break;
      const int it = ring[s];
      copy_tile(it, s, false);
      bulk_commit();
      bulk_wait_read0();   // the store has read the stage: hand it back to the loader
      mbar_arrive(&freed[s]);
      bulk_wait1();        // the previous store has completed: count it
      if (unrel >= 0) count_item(unrel);
      unrel = it;
    }
    bulk_wait_all();
    if (unrel >= 0) count_item(unrel);
    if (gave_up) atomicExch(a.status, 1);
    return;
  }

  // -------------------------------------------------------------------- compute warps (NG groups of NC threads)
  SweepArgs<float> sa{};
  sa.tw_fwd = G::TWS ? tws : a.tw_fwd;
  sa.tw_inv = G::TWS ? tws + G::TWF : a.tw_inv;
  sa.ekx = a.ekx;
  sa.ek2 = a.ek2;
  sa.scale_inv = 0;
  const int grp = tid / NC, lt = tid % NC;
  for (int k = grp;; k += NG) {
    const int s = k % S;
    // several groups: the stage may still serve an earlier item of another group; wait until the
    // loader has put this group's item into it (its k / S-th load), then for that load's phase
    bool ok = true;
    if constexpr (NG > 1) {
      ok = false;
      for (int w = 0; w < (1 << 22); ++w)
        if (issued[s] > k / S) {
          ok = true;
          break;
        }
    }
    ok = ok && mbar_wait_bounded(&full[s], (unsigned)(k / S) & 1u);
    if (!bar_and<NC>(ok)) {
      if (lt == 0) atomicExch(a.status, 1);
      break;
    }
    const int it = ring[s];
    if (it < 0) break;
    const int ph = it & 3, j = (it >> 2) & 511, z = (it >> 11) % L;
    V* sm = buf + (size_t)s * STAGE;
    if (ph == 1) {
      const int p = lt / TP, t = lt % TP;
      // the tile is [box k][row][x within box]
      auto addr = [&](int pos) { return sm + (pos / BOX) * (BOX * B) + p * BOX + (pos % BOX); };
      LayContig<L> lay;
      sweep_op_body<OP_FWD_K_INV, float, L, B, LayContig<L>, decltype(addr), true, (TP <= 32), G::TWS, NC>(
          sa, t, p, sm, lay, addr, j * B + p, z);
    } else {
      const int p = lt % B, t = lt / B;
      auto addr = [&](int pos) { return sm + pos * B + p; };
      LayStrided lay{B};
      if (ph == 0)
        sweep_op_body<OP_FWD, float, L, B, LayStrided, decltype(addr), true, false, G::TWS, NC>(sa, t, p, sm, lay,
                                                                                                addr, j * B + p, z);
      else
        sweep_op_body<OP_INV, float, L, B, LayStrided, decltype(addr), true, false, G::TWS, NC>(sa, t, p, sm, lay,
                                                                                                addr, j * B + p, z);
    }
    fence_async_smem();        // this thread's writes of the stage, before the TMA store reads it
    mbar_arrive(&empty[s]);
  }
}

// compute groups and stages of the grouped plane kernel: 512: three groups, five stages;
// 1024: two groups, three stages (a 1024-point stage is 70 KB)
template <int L> __host__ __device__ constexpr int plane_groups() { return L >= 1024 ? 2 : 3; }
template <int L> __host__ __device__ constexpr int plane_group_stages() { return L >= 1024 ? 3 : 5; }

template <int L> struct TmaPlaneLaunch {
  template <int NS, int NG> static int occupancy() {
    static int occ = -1;   // set on the first launch of the length, before any graph capture
    if (occ < 0) {
      cudaFuncSetAttribute(k_tma_plane<L, NS, NG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)TmaPlane<L, NS, NG>::SMEM);
      int nb = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tma_plane<L, NS, NG>, TmaPlane<L, NS, NG>::NT,
                                                    TmaPlane<L, NS, NG>::SMEM);
      occ = nb;
    }
    return occ;
  }
  // grid for a launch over `count` fields (the lag depends on it); cap > 0 limits the CTAs per SM
  template <int NS, int NG> static int grid(int count, int cap) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int items = 3 * count * L * TmaPlane<L, NS, NG>::Q;
    int per = occupancy<NS, NG>() > 0 ? occupancy<NS, NG>() : 1;
    if (cap > 0 && cap < per) per = cap;
    const int g = sms * per;
    return g > items ? items : g;
  }
  // Tickets in flight: each CTA holds up to S loaded items, the rest of a chunk and the item
  // being claimed.  A lag of 1.75 times that many tickets (in planes) keeps an item's inputs
  // complete by the time it is claimed and the data between the phases of a plane (2 lag
  // planes) in L2 (measured on GB300 at 256^3 with the L2 hints: 1.25x 154 us, 1.5x 150 us,
  // 1.75x 146.2 us and 301 MB of DRAM traffic, 2x 145.9 us and 365 MB, per launch).
  template <int NS, int NG> static int lag(int grid) {
    constexpr int per_plane = 3 * TmaPlane<L, NS, NG>::Q;
    return (7 * grid * (TmaPlane<L, NS, NG>::S + TmaPlane<L, NS, NG>::CHUNK + 1) / 4 + per_plane - 1) / per_plane + 1;
  }
  template <int NS, int NG> static cudaError_t run(TmaPlaneArgs& a, int cap, cudaStream_t s) {
    if (occupancy<NS, NG>() < 1) return cudaErrorInvalidConfiguration;
    const int g = grid<NS, NG>(a.count, cap);
    a.lag = lag<NS, NG>(g);
    k_tma_plane<L, NS, NG><<<g, TmaPlane<L, NS, NG>::NT, TmaPlane<L, NS, NG>::SMEM, s>>>(a);
    return cudaGetLastError();
  }
  // stages: 2 or 3 shared-memory stages; ctas_per_sm: 0 = as many as fit, else at most that many;
  // groups > 1: the grouped kernel (lengths >= 512; its own group and stage counts)
  static cudaError_t launch(TmaPlaneArgs& a, int stages, int ctas_per_sm, int groups, cudaStream_t s) {
    if constexpr (L >= 512) {
      if (groups > 1) return run<plane_group_stages<L>(), plane_groups<L>()>(a, ctas_per_sm, s);
    }
    if (groups > 1) return cudaErrorInvalidValue;
    return stages == 2 ? run<2, 1>(a, ctas_per_sm, s) : run<3, 1>(a, ctas_per_sm, s);
  }
};

}  // namespace gp

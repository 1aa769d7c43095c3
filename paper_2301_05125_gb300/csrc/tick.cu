// tick.cu -- the batched update as one persistent launch per tick (sm_103a).
//
// One cooperative kernel runs the deterministic update (Sec. 3.4 and Sec. 4:
// pilot rays, change measure, allocation, adaptive rays, blend) of every
// volume of a batch.  Its grid is as large as the GPU holds at once; the
// blocks walk the phases in order and meet at a grid-wide barrier between
// phases, since a phase reads what the previous one wrote for other probes
// (the 5x5x5 stencil, the allocation over all probes, the shadow jobs of
// other blocks' rays).  Within a phase the blocks take the volumes' work
// items -- the blocks of the ordinary kernels, "virtual blocks" -- in a
// grid-stride loop and run the ordinary kernels' device bodies (wave.cuh,
// phase.cuh) on them.  The allocation runs grid-wide over chunks of 2,048
// probes: each pass of the integer water-filling sums its chunks' partial
// results at a barrier, in the one-block kernel's arithmetic, so the rays
// per probe are the same integers.
//
// Every barrier wait gives up after a time limit (%globaltimer): the block
// that gives up sets the tick's status, every other block sees it at its
// next wait, and all return; the host reads the status (ADGI_ERR_TIMEOUT).
// Nothing waits without a limit, so a tick whose grid is not fully resident
// fails instead of hanging.
#include "adgi_internal.cuh"
#include "bvhbody.cuh"
#include "kernels.cuh"
#include "phase.cuh"
#include "wave.cuh"

namespace adgi {

namespace {

enum TickPhase {
    kPhClassify = 0,  // clip classes + this frame's blend plan (+ moving parts: triangles, Morton order)
    kPhHierarchy,     // moving parts: radix tree
    kPhBounds,        // moving parts: boxes, bottom up
    kPhPilot,         // pilot rays
    kPhPilotPrep,     // their shading: shadow jobs
    kPhPilotShadow,   // shadow rays
    kPhPilotFinish,   // direct light + multi-bounce term, pilot records
    kPhChangeState,   // q_v, q_r, triggers, octant sums G
    kPhChangeWeight,  // 5x5x5 sums of G -> W
    kPhAllocate,      // rays per probe and offsets (grid-wide)
    kPhMain,          // adaptive rays
    kPhMainPrep,
    kPhMainShadow,
    kPhMainFinish,
    kPhBlend,         // atlases
};
static_assert(kPhBlend + 1 == kTickPhases, "phase count");
static_assert(kTickRebuildMax == kSmallBuild, "a rebuilt moving part is sorted in one block");

// allocation partial sums per chunk (scratch rows of n_chunks entries)
enum TickRow { kRowPin = 0, kRowS, kRowG0, kRowG1, kRowSu0, kRowSu1, kRowCa, kRowCe, kRowLoc };
static_assert(kRowLoc + 1 == kTickScratch, "scratch rows");
constexpr int kPer = kTickChunk / kTickThreads;  // probes per thread in a chunk

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier number `idx`.  Returns false in every thread of the
// block when the tick has failed: this block's wait gave up, or another
// block's did (status set).  Thread 0 arrives and waits; the fences around
// the wait order every write of the grid before the barrier ahead of every
// read after it (the other threads meet thread 0 at the block barriers).
__device__ bool grid_sync(TickCtl* C, int idx)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire(&C->bar_gen);
        __threadfence();
        // the test hook: at barrier `stall` no block arrives, so it never completes
        const unsigned arrived = C->stall == idx ? 0u : atomicAdd(&C->bar_count, 1u) + 1u;
        if (arrived == gridDim.x) {
            if (idx < kTickStamps) C->t_bar[idx] = global_ns();
            C->bar_count = 0u;
            st_release(&C->bar_gen, gen + 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (ld_acquire(&C->bar_gen) == gen) {
                if (ld_acquire(reinterpret_cast<const unsigned*>(&C->status)) != 0u) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > C->limit_ns) {
                    atomicCAS(&C->status, 0, kTickTimedOut);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// the volume whose virtual blocks [row[i], row[i+1]) hold vb
__device__ __forceinline__ int volume_of(const uint32_t* row, int nv, uint32_t vb)
{
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row[mid] <= vb)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Threads [0, n) copy the object at src to dst in 8-byte words.  Through
// memcpy, not a word-typed pointer: stores through a pointer of another type
// would not count, for the optimizer, as writes to the struct's fields, so a
// field read after a copy could return a value cached from before it.
template <typename T>
__device__ __forceinline__ void copy_words(T* dst, const T* src, size_t bytes, int t, int n)
{
    static_assert(sizeof(T) % 8 == 0, "copied as 8-byte words");
    const char* s = reinterpret_cast<const char*>(src);
    char* d = reinterpret_cast<char*>(dst);
    for (size_t k = (size_t)t; k < bytes / 8; k += (size_t)n) {
        unsigned long long w;
        memcpy(&w, s + 8 * k, 8);
        memcpy(d + 8 * k, &w, 8);
    }
}

// Make volume i the block's current one (its parameters in shared memory).
// Called by every thread of the block with the same i.  The copy waits for
// every thread first: one may still be reading the previous volume's.
__device__ __forceinline__ void use_volume(const TickVol* __restrict__ vols, int i, TickVol& tv, int& cur)
{
    // one decision for the whole block (and a barrier: every thread is done
    // with the previous volume's parameters before they are overwritten)
    if (!__syncthreads_or(cur != i)) return;
    copy_words(&tv, vols + i, sizeof(TickVol), threadIdx.x, blockDim.x);
    __syncthreads();
    if (threadIdx.x == 0) cur = i;
    __syncthreads();
}

// sums over chunks [cb, ce) of row a: the total and the part before chunk c
__device__ __forceinline__ void chunk_sums(const unsigned long long* a, int cb, int ce, int c, uint64_t* red,
                                           uint64_t& tot, uint64_t& bef)
{
    if (threadIdx.x < 32) {
        uint64_t t = 0, b = 0;
        for (int k = cb + (int)threadIdx.x; k < ce; k += 32) {
            const uint64_t x = a[k];
            t += x;
            b += k < c ? x : 0ull;
        }
        t = warp_sum(t);
        b = warp_sum(b);
        if (threadIdx.x == 0) red[0] = t, red[1] = b;
    }
    __syncthreads();
    tot = red[0];
    bef = red[1];
    __syncthreads();
}

// The allocation of every volume (the one-block kernel k_allocate of
// update.cu, grid-wide): with clip classes only V_in probes take adaptive
// rays; E = (avg - 8) P - (m0 - 8) |V_in| extra rays beyond the floors are
// spread by W in proportional passes capped at rmax - m0, then one at a time
// in probe order (probes with W > 0 first).  Chunk c covers probes
// [2048 lc, 2048 lc + 2048) of its volume, thread t eight of them.  Returns
// false when a barrier wait failed.
__device__ bool tick_allocate(const TickVol* __restrict__ vols, const int* __restrict__ cvol, int n_chunks,
                              unsigned long long* scr, TickCtl* C, int& bar, TickVol& tv, int& cur)
{
    __shared__ uint64_t red[66];
    __shared__ uint64_t o_erem[kTickOwn], o_su[kTickOwn];
    __shared__ int o_act[kTickOwn];  // 1 proportional passes, 2 remainder rounds, 0 done
    __shared__ int o_modeA[kTickOwn];
    unsigned long long* row[kTickScratch];
    for (int r = 0; r < kTickScratch; ++r) row[r] = scr + (size_t)r * n_chunks;
    const int nown = (n_chunks - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // chunks of this block
    auto chunk = [&](int k) { return (int)blockIdx.x + k * (int)gridDim.x; };
    // thread range [c0, c1) of chunk c of the current volume, and the volume's chunks [cb, ce)
    auto range = [&](int c, int& c0, int& c1, int& cb, int& ce) {
        const int P = tv.w.V.P, lc = c - tv.chunk0;
        c0 = min(P, lc * kTickChunk + (int)threadIdx.x * kPer);
        c1 = min(P, c0 + kPer);
        cb = tv.chunk0;
        ce = tv.chunk0 + (P + kTickChunk - 1) / kTickChunk;
    };
    auto vin = [&](int p) { return tv.cls[p] == 2; };
    auto w_of = [&](int p) -> uint32_t { return vin(p) ? tv.C.W[p] : 0u; };

    // 1. V_in counts and weight sums; the extras start at 0 (at the cap outside V_in)
    for (int k = 0; k < nown; ++k) {
        const int c = chunk(k);
        use_volume(vols, cvol[c], tv, cur);
        int c0, c1, cb, ce;
        range(c, c0, c1, cb, ce);
        const uint32_t cap = (uint32_t)(tv.rmax - tv.m0);
        uint64_t pin = 0, s = 0;
        for (int p = c0; p < c1; ++p) {
            const bool in = vin(p);
            pin += in ? 1u : 0u;
            s += in ? tv.C.W[p] : 0u;
            tv.n[p] = in ? 0u : cap;
        }
        block_sum2(pin, s, red);
        if (threadIdx.x == 0) row[kRowPin][c] = pin, row[kRowS][c] = s;
    }
    if (!grid_sync(C, bar++)) return false;
    // 2. E per volume; W = 0 everywhere: uniform over V_in, remainder to the lowest V_in ranks
    for (int k = 0; k < nown; ++k) {
        const int c = chunk(k);
        use_volume(vols, cvol[c], tv, cur);
        int c0, c1, cb, ce;
        range(c, c0, c1, cb, ce);
        const uint32_t cap = (uint32_t)(tv.rmax - tv.m0);
        uint64_t Pin, rank0, S, s_bef;
        chunk_sums(row[kRowPin], cb, ce, c, red, Pin, rank0);
        chunk_sums(row[kRowS], cb, ce, c, red, S, s_bef);
        uint64_t E = (uint64_t)(tv.avg - 8) * (uint64_t)tv.w.V.P - (uint64_t)(tv.m0 - 8) * Pin;
        if (E > Pin * cap) E = Pin * cap;
        if (S == 0) {
            const uint64_t q = Pin ? E / Pin : 0, r = Pin ? E % Pin : 0;
            uint64_t tpin = 0;
            for (int p = c0; p < c1; ++p) tpin += vin(p) ? 1u : 0u;
            uint64_t tot;
            uint64_t rank = rank0 + block_exscan(tpin, red, &tot);
            for (int p = c0; p < c1; ++p) {
                if (!vin(p)) continue;
                tv.n[p] = (uint32_t)(q + (rank < r ? 1u : 0u));
                ++rank;
            }
        }
        if (threadIdx.x == 0) {
            o_erem[k] = E;
            o_su[k] = cap > 0u ? S : 0u;
            o_act[k] = S == 0 ? 0 : 1;
        }
        __syncthreads();
    }
    // 3. proportional passes: SU = the weight of the probes below their cap
    for (int it = 0; it < kTickPasses; ++it) {
        for (int k = 0; k < nown; ++k) {
            if (o_act[k] != 1) continue;
            if (o_su[k] == 0 || o_erem[k] == 0) {
                __syncthreads();
                if (threadIdx.x == 0) o_act[k] = 2;
                __syncthreads();
                continue;
            }
            const int c = chunk(k);
            use_volume(vols, cvol[c], tv, cur);
            int c0, c1, cb, ce;
            range(c, c0, c1, cb, ce);
            const uint32_t cap = (uint32_t)(tv.rmax - tv.m0);
            const uint64_t Erem = o_erem[k], SU = o_su[k];
            const uint64_t inv = 0xFFFFFFFFFFFFFFFFull / SU;
            uint64_t G = 0, su = 0;
            for (int p = c0; p < c1; ++p) {
                const uint32_t w = w_of(p), e = tv.n[p];
                if (w == 0u || e >= cap) continue;
                const uint64_t share = div_by(Erem * (uint64_t)w, SU, inv);
                const uint64_t room = cap - e;
                const uint64_t a = share < room ? share : room;
                tv.n[p] = e + (uint32_t)a;
                G += a;
                if (a < room) su += w;
            }
            block_sum2(G, su, red);
            if (threadIdx.x == 0) {
                row[(it & 1) ? kRowG1 : kRowG0][c] = G;
                row[(it & 1) ? kRowSu1 : kRowSu0][c] = su;
                C->pass_flag[it] = 1u;
            }
        }
        if (!grid_sync(C, bar++)) return false;
        if (*reinterpret_cast<volatile unsigned*>(&C->pass_flag[it]) == 0u) break;  // no chunk took part
        for (int k = 0; k < nown; ++k) {
            if (o_act[k] != 1) continue;
            const int c = chunk(k);
            use_volume(vols, cvol[c], tv, cur);
            int c0, c1, cb, ce;
            range(c, c0, c1, cb, ce);
            uint64_t Gt, Gb, St, Sb;
            chunk_sums(row[(it & 1) ? kRowG1 : kRowG0], cb, ce, c, red, Gt, Gb);
            chunk_sums(row[(it & 1) ? kRowSu1 : kRowSu0], cb, ce, c, red, St, Sb);
            if (threadIdx.x == 0) {
                if (Gt == 0) {
                    o_act[k] = 2;
                } else {
                    o_erem[k] -= Gt;
                    o_su[k] = St;
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < nown; ++k)
            if (o_act[k] == 1) o_act[k] = 2;  // the pass bound was reached
    __syncthreads();
    // 4. remainder: one ray each, probe order, probes with W > 0 first
    for (int j = 0; j < (1 << 20); ++j) {
        for (int k = 0; k < nown; ++k) {
            if (o_act[k] != 2) continue;
            if (o_erem[k] == 0) {
                __syncthreads();
                if (threadIdx.x == 0) o_act[k] = 0;
                __syncthreads();
                continue;
            }
            const int c = chunk(k);
            use_volume(vols, cvol[c], tv, cur);
            int c0, c1, cb, ce;
            range(c, c0, c1, cb, ce);
            const uint32_t cap = (uint32_t)(tv.rmax - tv.m0);
            uint64_t ca = 0;
            for (int p = c0; p < c1; ++p)
                if (w_of(p) > 0u && tv.n[p] < cap) ++ca;
            ca = block_sum(ca, red);
            if (threadIdx.x == 0) {
                row[kRowCa][c] = ca;
                C->rem_flag[j & 1] = 1u;
            }
        }
        if (!grid_sync(C, bar++)) return false;
        if (*reinterpret_cast<volatile unsigned*>(&C->rem_flag[j & 1]) == 0u) break;
        for (int k = 0; k < nown; ++k) {
            if (o_act[k] != 2) continue;
            const int c = chunk(k);
            use_volume(vols, cvol[c], tv, cur);
            int c0, c1, cb, ce;
            range(c, c0, c1, cb, ce);
            const uint32_t cap = (uint32_t)(tv.rmax - tv.m0);
            uint64_t cat, cab;
            chunk_sums(row[kRowCa], cb, ce, c, red, cat, cab);
            const bool modeA = cat > 0;
            uint64_t ce_n = 0;
            for (int p = c0; p < c1; ++p)
                if (tv.n[p] < cap && (!modeA || w_of(p) > 0u)) ++ce_n;
            ce_n = block_sum(ce_n, red);
            if (threadIdx.x == 0) {
                row[kRowCe][c] = ce_n;
                o_modeA[k] = modeA ? 1 : 0;
            }
            __syncthreads();
        }
        if (!grid_sync(C, bar++)) return false;
        // every block has read this round's flag: clear it for round j + 2
        if (blockIdx.x == 0 && threadIdx.x == 0) C->rem_flag[j & 1] = 0u;
        for (int k = 0; k < nown; ++k) {
            if (o_act[k] != 2) continue;
            const int c = chunk(k);
            use_volume(vols, cvol[c], tv, cur);
            int c0, c1, cb, ce;
            range(c, c0, c1, cb, ce);
            const uint32_t cap = (uint32_t)(tv.rmax - tv.m0);
            uint64_t tot, bef;
            chunk_sums(row[kRowCe], cb, ce, c, red, tot, bef);
            if (tot == 0) {
                if (threadIdx.x == 0) o_act[k] = 0;
                __syncthreads();
                continue;
            }
            const bool modeA = o_modeA[k] != 0;
            const uint64_t Erem = o_erem[k];
            uint64_t mine = 0;
            for (int p = c0; p < c1; ++p)
                if (tv.n[p] < cap && (!modeA || w_of(p) > 0u)) ++mine;
            uint64_t t2;
            uint64_t pre = bef + block_exscan(mine, red, &t2);
            for (int p = c0; p < c1; ++p) {
                if (tv.n[p] < cap && (!modeA || w_of(p) > 0u)) {
                    if (pre < Erem) tv.n[p] += 1u;
                    ++pre;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) o_erem[k] = Erem - (tot < Erem ? tot : Erem);
            __syncthreads();
        }
    }
    // 5. rays per probe (the floor plus the extra) and the adaptive-ray offsets
    auto rays_of = [&](int p) -> uint32_t {
        if (vin(p)) return (uint32_t)tv.m0 + tv.n[p];
        return tv.cls[p] == 1 ? 8u : 0u;
    };
    for (int k = 0; k < nown; ++k) {
        const int c = chunk(k);
        use_volume(vols, cvol[c], tv, cur);
        int c0, c1, cb, ce;
        range(c, c0, c1, cb, ce);
        uint64_t loc = 0;
        for (int p = c0; p < c1; ++p) {
            const uint32_t np = rays_of(p);
            loc += np > 8u ? np - 8u : 0u;
        }
        loc = block_sum(loc, red);
        if (threadIdx.x == 0) row[kRowLoc][c] = loc;
    }
    if (!grid_sync(C, bar++)) return false;
    for (int k = 0; k < nown; ++k) {
        const int c = chunk(k);
        use_volume(vols, cvol[c], tv, cur);
        int c0, c1, cb, ce;
        range(c, c0, c1, cb, ce);
        uint64_t tot, bef;
        chunk_sums(row[kRowLoc], cb, ce, c, red, tot, bef);
        uint64_t loc = 0;
        for (int p = c0; p < c1; ++p) {
            const uint32_t np = rays_of(p);
            loc += np > 8u ? np - 8u : 0u;
        }
        uint64_t t2;
        uint64_t pre = bef + block_exscan(loc, red, &t2);
        for (int p = c0; p < c1; ++p) {
            const uint32_t np = rays_of(p), a = (uint32_t)pre, e = a + (np > 8u ? np - 8u : 0u);
            tv.off[p] = a;
            for (uint32_t q = (a + 31u) / 32u; 32u * q < e; ++q) tv.w.chunk_p[q] = (uint32_t)p;  // chunks starting here
            pre = e;
            tv.n[p] = np;
        }
        if (threadIdx.x == 0 && c == ce - 1) tv.off[tv.w.V.P] = (uint32_t)tot;
        __syncthreads();
    }
    return true;
}

__global__ void __launch_bounds__(kTickThreads, 4) k_tick(const TickVol* __restrict__ vols, int nv,
                                                       const uint32_t* __restrict__ pre,
                                                       const int* __restrict__ cvol, int n_chunks,
                                                       unsigned long long* scr, TickCtl* C,
                                                       const int* __restrict__ rebuild, int any_rebuild)
{
    __shared__ __align__(16) TickVol tv;
    __shared__ int cur;
    // The ray phases run per warp, with no block barrier between a warp's
    // work items (a block would otherwise wait for its slowest warp's
    // rays); a warp reads its volume's ray parameters (TickWave) straight
    // from the read-only table.
    const unsigned lane = threadIdx.x & 31u;
    if (threadIdx.x == 0) cur = -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) C->t_start = global_ns();
    __syncthreads();
    int bar = 0;
    for (int ph = 0; ph < kTickPhases; ++ph) {
        if (!any_rebuild && (ph == kPhHierarchy || ph == kPhBounds)) continue;  // (and their barriers)
        if (ph == kPhPilotShadow || ph == kPhMainShadow) {
            // every volume's shadow jobs, in rounds of 32 consecutive jobs
            // of one list (one job a lane); the rounds of all lists in
            // volume order form one sequence, and each warp takes the next
            // round from a grid-wide counter, so warps that drew short rays
            // take more rounds and all end together
            unsigned* next = &C->next_item[ph == kPhPilotShadow ? 2 : 3];
            int i = 0;
            unsigned first = 0;  // the first round of volume i
            unsigned total = min(*vols[0].w.Wk.job_count, vols[0].w.Wk.job_cap);
            for (;;) {
                unsigned g = 0;
                if (lane == 0) g = atomicAdd(next, 1u);
                g = __shfl_sync(0xFFFFFFFFu, g, 0);
                while (i < nv && g >= first + (total + 31u) / 32u) {  // rounds are taken in increasing order
                    first += (total + 31u) / 32u;
                    if (++i < nv) total = min(*vols[i].w.Wk.job_count, vols[i].w.Wk.job_cap);
                }
                if (i >= nv) break;
                const TickWave& T = vols[i].w;
                const unsigned r = g - first, j = 32u * r + lane;
                if (r == 0 && lane == 0) atomicAdd(T.Wk.shadow_ctr, (unsigned long long)total);
                if (j < total) shadow_job<true>(T.FD->L, T.S, T.Wk.jobs, T.Wk.job_light, T.Wk.vis, j);
                __syncwarp();  // the lanes take the next round together
            }
            __syncthreads();
        } else if (ph == kPhPilot || ph == kPhMain) {
            // warp items: 32 pilot rays of one octant, or 32 adaptive rays,
            // each warp taking the next item from a grid-wide counter
            const uint32_t* row = pre + (size_t)ph * (nv + 1);
            const uint32_t total = row[nv];
            unsigned* next = &C->next_item[ph == kPhPilot ? 0 : 1];
            for (;;) {
                uint32_t vw = 0;
                if (lane == 0) vw = atomicAdd(next, 1u);
                vw = __shfl_sync(0xFFFFFFFFu, vw, 0);
                if (vw >= total) break;
                const int i = volume_of(row, nv, vw);
                const TickWave& T = vols[i].w;
                const uint32_t lw = vw - row[i];
                if (ph == kPhPilot)
                    pilot_trace_body<true>(T.V, T.FD, T.S, T.pil_hit, (int)(32u * lw) + lane);
                else
                    main_trace_warp_body<true>(T.V, T.FD, T.S, T.off, T.sf, T.V.R_main, T.m_hit, lw, T.chunk_p);
                // The lanes leave an item at different times (independent
                // thread scheduling); they start the next one together, since
                // its warp shuffles need all of them.
                __syncwarp();
            }
            __syncthreads();
        } else if (ph == kPhAllocate) {
            if (!tick_allocate(vols, cvol, n_chunks, scr, C, bar, tv, cur)) return;
        } else {
            const uint32_t* row = pre + (size_t)ph * (nv + 1);
            const uint32_t total = row[nv];
            for (uint32_t vb = blockIdx.x; vb < total; vb += gridDim.x) {
                const int i = volume_of(row, nv, vb);
                use_volume(vols, i, tv, cur);
                const uint32_t lb = vb - row[i];
                const VolConst& V = tv.w.V;
                const bool rb = rebuild[i] != 0;
                switch (ph) {
                case kPhClassify: {
                    const uint32_t nc = ((uint32_t)V.P + kTickThreads - 1) / kTickThreads;
                    const uint32_t np = (uint32_t)max(V.rays_max - kPilots, 0);
                    const uint32_t nf = tv.nd > 0 && tv.nd <= kTickRebuildMax
                                            ? ((uint32_t)tv.nd + kTickThreads - 1) / kTickThreads : 0u;
                    if (lb < nc) {
                        classify_body(V, tv.w.FD, tv.lut_c, tv.cls, lb);
                    } else if (lb < nc + np) {
                        blend_plan_body(V, tv.w.FD, tv.w.sf, tv.B.plan, lb - nc);
                    } else if (lb < nc + np + nf) {  // the moving triangles in original order (shading)
                        if (rb)
                            fill_orig_body(tv.verts, tv.idx, tv.dlist, tv.nd, tv.nv, tv.tri_orig,
                                           (int)(lb - nc - np) * kTickThreads + (int)threadIdx.x);
                    } else if (rb) {  // the moving part's Morton order, sorted by this block (in global memory)
                        morton_small_body(tv.verts, tv.idx, tv.dlist, tv.nd, tv.nv, tv.tri_in, tv.keys, tv.vals,
                                          const_cast<float4*>(tv.w.S.tri_v) + 3 * (size_t)tv.tri_off, tv.w.S.err,
                                          tv.sort_k, tv.sort_v);
                        for (int k = threadIdx.x; k < tv.nd; k += blockDim.x) tv.flags[k] = 0;
                    }
                    break;
                }
                case kPhHierarchy:
                    if (rb)
                        hierarchy_body(tv.keys, tv.nd, const_cast<BNode*>(tv.w.S.nodes) + tv.node_off, tv.par_int,
                                       tv.par_leaf, (int)lb * kTickThreads + (int)threadIdx.x, tv.node_off, tv.tri_off);
                    break;
                case kPhBounds:
                    if (rb)
                        bounds_body(tv.w.S.tri_v + 3 * (size_t)tv.tri_off, tv.nd, const_cast<BNode*>(tv.w.S.nodes) + tv.node_off,
                                    tv.par_int, tv.par_leaf, tv.flags, tv.eps, tv.w.S.err,
                                    (int)lb * kTickThreads + (int)threadIdx.x, tv.node_off, tv.tri_off);
                    break;
                case kPhPilotPrep: {
                    const RaySet Rs{0, (uint32_t)V.P * kPilots, nullptr, nullptr, DynRays{}};
                    shade_prep_body<true>(V, tv.w.FD, tv.w.S, Rs, tv.w.pil_hit, tv.w.Wk.vis, tv.w.Wk.jobs, tv.w.Wk.job_light,
                                          tv.w.Wk.job_count, tv.w.Wk.job_cap, lb);
                    break;
                }
                case kPhPilotFinish: {
                    const RaySet Rs{0, (uint32_t)V.P * kPilots, nullptr, nullptr, DynRays{}};
                    shade_finish_body<true>(V, tv.w.FD, tv.w.S, Rs, tv.w.pil_hit, tv.w.Wk.vis, tv.B.irr, tv.B.dep, tv.pil_rec,
                                            tv.pil_lum, lb);
                    break;
                }
                case kPhChangeState:
                    change_state_body(V, tv.w.FD, tv.C, lb);
                    break;
                case kPhChangeWeight:
                    change_weight_body<true>(V, tv.w.FD, tv.C, lb);
                    break;
                case kPhMainPrep: {
                    const RaySet Rs{1, V.R_main, tv.off, tv.w.sf, DynRays{}};
                    shade_prep_body<true>(V, tv.w.FD, tv.w.S, Rs, tv.w.m_hit, tv.w.Wk.vis, tv.w.Wk.jobs, tv.w.Wk.job_light,
                                          tv.w.Wk.job_count, tv.w.Wk.job_cap, lb);
                    break;
                }
                case kPhMainFinish: {
                    const RaySet Rs{1, V.R_main, tv.off, tv.w.sf, DynRays{}};
                    shade_finish_body<true>(V, tv.w.FD, tv.w.S, Rs, tv.w.m_hit, tv.w.Wk.vis, tv.B.irr, tv.B.dep, tv.m_rec,
                                            nullptr, lb);
                    break;
                }
                case kPhBlend:
                    blend_body<true>(V, tv.w.FD, tv.B, lb, kTickBlendWarps);
                    break;
                default:
                    break;
                }
                __syncthreads();
            }
        }
        // the shadow-job counters: cleared before each shading's prep step
        if ((ph == kPhClassify || ph == kPhPilotFinish) && blockIdx.x == 0) {
            for (int i = threadIdx.x; i < nv; i += blockDim.x) {
                *vols[i].w.Wk.job_count = 0u;
                if (ph == kPhClassify) *vols[i].w.Wk.shadow_ctr = 0ull;
            }
        }
        if (ph + 1 < kTickPhases && !grid_sync(C, bar++)) return;
    }
}

}  // namespace

void tick_phase_blocks(const VolConst& V, uint32_t R_main, int nd, uint32_t counts[kTickPhases])
{
    const uint32_t P = (uint32_t)V.P, T = kTickThreads, M = (uint32_t)std::max(V.rays_max - kPilots, 0);
    for (int i = 0; i < kTickPhases; ++i) counts[i] = 0;
    counts[kPhClassify] = (P + T - 1) / T + M;
    if (nd > 0 && nd <= kTickRebuildMax) {  // the moving part's rebuild: fill + one sorting block, tree, boxes
        const uint32_t n = (uint32_t)nd;
        counts[kPhClassify] += (n + T - 1) / T + 1;
        counts[kPhHierarchy] = n > 1 ? (n - 1 + T - 1) / T : 0;
        counts[kPhBounds] = n > 1 ? (n + T - 1) / T : 0;
    }
    counts[kPhPilot] = (P + 31) / 32 * kPilots;  // warp items: 32 probes x one octant
    counts[kPhPilotPrep] = counts[kPhPilotFinish] = (P * kPilots + T - 1) / T;
    counts[kPhChangeState] = counts[kPhChangeWeight] = (P + T - 1) / T;
    counts[kPhMainPrep] = counts[kPhMainFinish] = (R_main + T - 1) / T;
    counts[kPhMain] = (R_main + 31) / 32;  // warp items of 32 rays
    counts[kPhBlend] = (P + kTickBlendWarps - 1) / kTickBlendWarps;  // one warp per probe tile
}

// Kept small: the shared-memory carve-out takes from the L1 cache that the
// traversal phases read the tree, the triangles and their stacks through.
size_t tick_smem_bytes(const VolConst& V)
{
    const size_t blend = (size_t)blend_layout(V.Ti, V.Td).total * kTickBlendWarps;
    return std::max(blend, blend_plan_smem(V));
}

unsigned tick_grid_blocks(size_t smem)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (raise_smem_limit((const void*)k_tick, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tick, kTickThreads, smem) != cudaSuccess) return 0;
    return sms > 0 && per > 0 ? (unsigned)(sms * per) : 0u;
}

cudaError_t launch_tick(const TickVol* vols, int nv, const uint32_t* pre, const int* cvol, int n_chunks,
                        unsigned long long* scratch, TickCtl* ctl, const int* rebuild, int any_rebuild, unsigned grid,
                        size_t smem, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(kTickThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every block resident at once
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_tick, vols, nv, pre, cvol, n_chunks, scratch, ctl, rebuild, any_rebuild);
    count_launches(1);
    return e;
}

}  // namespace adgi

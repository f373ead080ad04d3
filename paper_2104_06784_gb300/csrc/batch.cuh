// batch.cuh -- the ensemble launch: every stage of every member simulation in
// one cooperative launch of resident CTAs (batch_persistent_kernel), with a
// bounded grid barrier (grid_meet) between the classification and the stage
// and between the stage and the next classification.  The stage arithmetic is
// stage.cuh's stage_tile; the classification is its classify_strip on the
// first stage of a call whose mass bits are not known, else the mass bits.
#pragma once
#include <cuda_runtime.h>

#include "stage.cuh"

namespace moses {
// Ensemble form: one launch covers many simulations.  Each simulation keeps
// its own control block, so its own time and time step.  The classification
// appends the wet tiles of every simulation, as (simulation, tile), to one
// list; the stage runs that list, each CTA copying its tile's simulation
// arguments into shared memory.
struct BatchTile {
    int sim, bx, by;
};
struct BatchStrip {
    int sim, sx, sy;
};

template <typename T>
__device__ __forceinline__ void copy_args(StageArgs<T> &dst, const StageArgs<T> *src)
{
    // cooperative copy of a descriptor (plain 4-byte words)
    const int *s = reinterpret_cast<const int *>(src);
    int *d = reinterpret_cast<int *>(&dst);
    for (int q = threadIdx.x; q < (int)(sizeof(StageArgs<T>) / 4); q += blockDim.x) d[q] = s[q];
}

// ---- the ensemble as one persistent launch -----------------------------------
// A cooperative launch whose CTAs all stay resident runs every stage of every
// member for all the steps of a call.  Between the phases of a stage the CTAs
// meet on a grid barrier in device memory: arrivals are counted, and the CTA
// that arrives last runs the phase's closing work with all its threads, then
// opens the next generation.  Every wait is bounded (0.5 s by the global
// timer, and 2^26 tries): a CTA that gives up raises `fail`, every CTA that
// sees it leaves the launch, and the host returns MOSES_ETIMEOUT.
struct GridSync {
    unsigned int count;   // arrivals in the current generation
    unsigned int gen;     // generation, advanced by the last arrival
    unsigned int expect;  // arrivals that close a generation: the grid (testing: one more, so that every wait runs out)
    int fail;             // a wait gave up, or a classification's copy wait did
};

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }
// a load that orders nothing: the barrier's waits poll with it (an acquiring
// load would also drop the SM's L1, under the feet of the CTAs that still work)
__device__ __forceinline__ unsigned int ld_relaxed_gpu(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All CTAs meet; the last to arrive runs closing() first.  False: the launch
// failed (a wait ran out here or elsewhere): the caller leaves.
template <typename F>
__device__ bool grid_meet(GridSync *g, const F &closing)
{
    __shared__ int s_state;  // 0: waited, 1: arrived last, 2: gave up
    __shared__ int s_ok;     // the launch goes on (one thread reads the fail word for the CTA)
    __syncthreads();
    if (threadIdx.x == 0) {
        // the generation is read before this CTA arrives (it cannot advance
        // before then); the fence releases the CTA's writes before its arrival
        const unsigned int gen = ld_relaxed_gpu(&g->gen);
        __threadfence();
        const unsigned int n = atomicAdd(&g->count, 1u) + 1u;
        int state = n == ld_relaxed_gpu(&g->expect) ? 1 : 0;
        if (state == 0) {
            const unsigned long long t0 = global_ns();
            for (int it = 0;; ++it) {
                if (ld_relaxed_gpu(&g->gen) != gen) break;
                if (ld_volatile(&g->fail) || it >= (1 << 26) ||
                    ((it & 255) == 255 && global_ns() - t0 > 500000000ull)) {
                    atomicExch(&g->fail, 1);
                    state = 2;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();  // acquires what the other CTAs wrote before they arrived
        s_state = state;
    }
    __syncthreads();
    const int state = s_state;
    if (state == 1) {
        closing();
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicExch(&g->count, 0u);
            __threadfence();
            atomicAdd(&g->gen, 1u);
        }
    }
    if (threadIdx.x == 0) s_ok = state != 2 && ld_volatile(&g->fail) == 0;
    __syncthreads();
    const bool ok = s_ok != 0;
    __syncthreads();  // s_state and s_ok are written again at the next meeting
    return ok;
}

// One ensemble launch: the stage descriptors of every member (stage 1 from U
// to U*, stage 2 from U* back to U with the Heun average), the strips of the
// data classification, every tile of every member (tile_sim: its member;
// tile_base: a member's first tile), the shared wet-tile list, the barrier,
// and the steps to run.  from_data: 1 when the members' mass bits are not
// known yet (the first stage of the first step then classifies from the data
// and writes them); the launch clears it.  nstages: stages to run (2 per
// step; 1 runs the first stage alone, for timing the tile shapes).
template <typename T>
struct BatchRun {
    const StageArgs<T> *args1, *args2;
    int nsim;
    const BatchStrip *strips;
    int nstrips;
    const int *tile_sim, *tile_base;
    int ntiles;
    BatchTile *list;
    unsigned int *list_n;
    GridSync *sync;
    int *from_data;
    int nstages;
};

// The mass-bit classification of one stage over every tile of every member,
// in chunks of blockDim.x tiles per CTA (as classify_flags_kernel does for one
// simulation), with the chunk's dry tiles zero-written by the CTA's warps.
template <typename T, int TY>
__device__ void classify_batch_bits(const BatchRun<T> &r, const StageArgs<T> *args, int *s_list, unsigned int &s_n)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const T z[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    for (int base = blockIdx.x * blockDim.x; base < r.ntiles; base += gridDim.x * blockDim.x) {
        if (tid == 0) s_n = 0u;
        __syncthreads();
        const int idx = base + tid;
        if (idx < r.ntiles) {
            const int k = r.tile_sim[idx];
            const StageArgs<T> &a = args[k];
            const int t = idx - r.tile_base[k];
            const int gx = (a.nx + 31) / 32, gy = (a.ny + TY - 1) / TY, bx = t % gx, ty = t / gx;
            const unsigned char known = a.zk ? a.zk[t] : 0;
            bool w = wet_from_bits(a.mb_in, bx, ty, gx, gy);
            if (a.mb_n) w |= (a.mb_n[t] & MB_ANY) != 0;
            const bool inf = on_inflow_side(a, bx, ty, gx, gy);
            w |= inf;
            if (w) r.list[atomicAdd(&r.list_n[0], 1u)] = BatchTile{k, bx, ty};
            if (!w) a.mb_out[t] = 0;
            if (!keep_tile(a, w, inf, t, known)) s_list[atomicAdd(&s_n, 1u)] = idx;
            if (a.stage == 1 && t == 0) {
                const double dt = dt_from(a.ctl, a.ph, __longlong_as_double((long long)a.ctl->amax));
                first_stage_clock(a, a.ctl->t, dt);
            }
        }
        __syncthreads();
        const int nrows = (int)s_n * TY;
        for (int rr = warp; rr < nrows; rr += nw) {
            const int idx2 = s_list[rr / TY], k = r.tile_sim[idx2];
            const StageArgs<T> &a = args[k];
            const int t = idx2 - r.tile_base[k], gx = (a.nx + 31) / 32;
            const int i = (t % gx) * 32 + lane, j = (t / gx) * TY + rr % TY;
            if (i >= a.nx || j >= a.ny) continue;
            const Ctl *ctl = a.ctl;
            const double tg = a.stage == 1 ? ctl->t + dt_from(ctl, a.ph, __longlong_as_double((long long)ctl->amax))
                                           : ctl->t + ctl->dt;
            const long long g = cell_index(i, j, a.pitch);
            store6(a.Uout, a.plane, g, z);
            if constexpr (sizeof(T) == 4) {
                a.Rout[g] = 0.0f;
                a.Rout[a.plane + g] = 0.0f;
            }
            write_ghosts(a.Uout, a.geo, a, i, j, z, tg);
        }
        __syncthreads();
    }
}

// The ensemble launch (BatchRun): per stage, the classification (from the
// data on the first stage of the call when the mass bits are not known,
// else from the bits), a meeting, the stage on the listed tiles, a meeting
// whose closing empties the list and, after a step's last stage, ends the
// step of every member.  The classification's strip buffers and the stage
// kernel's tile buffers share the dynamic shared memory.
template <typename T, int TY>
__global__ void __launch_bounds__(32 * TY, (sizeof(T) == 4 ? 768 : 512) / (32 * TY))
    batch_persistent_kernel(const BatchRun<T> r)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ StageArgs<T> sa;
    __shared__ int s_list[32 * TY];
    __shared__ unsigned int s_n;
    __shared__ unsigned int s_word;  // a word of device memory one thread read for the CTA
    ClassifySmem<T> &cs = *reinterpret_cast<ClassifySmem<T> *>(smem_raw);
    // (words of device memory that every thread needs are read by one thread:
    // a read per thread of one address serialises in L2)
    if (threadIdx.x == 0) s_word = (unsigned int)ld_volatile(r.from_data);
    __syncthreads();
    const bool data = s_word != 0u;  // read by every CTA before the first meeting clears it
    for (int q = 0; q < r.nstages; q++) {
        const bool second = q & 1;
        const StageArgs<T> *args = second ? r.args2 : r.args1;
        // ---- classification ----
        if (q == 0 && data) {
            bool ok = true;
            for (int w = blockIdx.x; w < r.nstrips && ok; w += gridDim.x) {
                const BatchStrip st = r.strips[w];
                // this thread's generic accesses to cs (the strip before) come
                // before the bulk copies that reuse it
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();  // sa and cs are free
                copy_args(sa, args + st.sim);
                __syncthreads();
                const int sim = st.sim;
                ok = classify_strip<T, TY>(sa, st.sx, st.sy, (sa.nx + 31) / 32, cs, [&](int tx, int ty) {
                    r.list[atomicAdd(&r.list_n[0], 1u)] = BatchTile{sim, tx, ty};
                });
            }
            if (!ok && threadIdx.x == 0) atomicExch(&r.sync->fail, 1);
        } else {
            classify_batch_bits<T, TY>(r, args, s_list, s_n);
        }
        if (!grid_meet(r.sync, [&] {
                if (q == 0 && threadIdx.x == 0) *r.from_data = 0;
            }))
            return;
        // ---- the stage on the listed tiles ----
        if (threadIdx.x == 0) s_word = ld_acquire_gpu(&r.list_n[0]);
        __syncthreads();
        const unsigned int n = s_word;
        for (unsigned int w = blockIdx.x; w < n; w += gridDim.x) {
            const BatchTile t = r.list[w];
            __syncthreads();  // the previous tile is done with sa
            copy_args(sa, args + t.sim);
            __syncthreads();
            stage_tile<T, 32, TY>(sa, t.bx, t.by, 0u);
        }
        if (!grid_meet(r.sync, [&] {
                if (threadIdx.x == 0) r.list_n[0] = 0u;
                if (second)
                    for (int k = threadIdx.x; k < r.nsim; k += blockDim.x) end_step(r.args2[k]);
            }))
            return;
    }
}

}  // namespace moses

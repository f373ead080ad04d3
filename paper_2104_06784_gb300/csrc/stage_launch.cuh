// stage_launch.cuh -- launchers of the templated stage kernels (stage.cuh,
// and the ensemble kernel of batch.cuh),
// shared by the two precision forms; stage_f64.cu and stage_f32.cu each
// instantiate them for one element type (one translation unit per type, so
// that the two compile in parallel).
#pragma once
#include <cuda_runtime.h>

#include "batch.cuh"
#include "stage.cuh"

namespace moses {
namespace {

template <typename T, int TX, int TY, bool REC = false, bool VIS = false, bool CU = false, bool WENO = false,
          bool KM = false>
int launch_tile(const StageArgs<T> &a, cudaStream_t st)
{
    constexpr size_t smem = stage_smem_bytes<T, TX, TY, VIS, KM>();
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(stage_kernel<T, TX, TY, REC, VIS, CU, WENO, KM>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return -1;
        attr_set[dev] = true;
    }
    const dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
    stage_kernel<T, TX, TY, REC, VIS, CU, WENO, KM><<<grid, TX * TY, smem, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

// The stepping launches of the plain form: classify_kernel over every tile
// (classify_flags_kernel where the input's mass bits are known, and in a
// combining stage), then stage_kernel_list on a grid of resident CTAs over
// the listed tiles (P2: two threads per cell).
template <typename T, int TX, int TY, bool REC = false, bool KM = false, bool P2 = false>
int launch_tile_list(const StageArgs<T> &a, cudaStream_t st)
{
    constexpr int NTH = TX * TY * (P2 ? 2 : 1);
    constexpr size_t smem = stage_smem_bytes<T, TX, TY, false, KM>();
    static int resident[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return -1;
    if (!resident[dev]) {
        int per_sm = 0, n_sm = 0;
        if (cudaFuncSetAttribute(stage_kernel_list<T, TX, TY, REC, KM, P2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_kernel_list<T, TX, TY, REC, KM, P2>, NTH, smem) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1 || n_sm < 1)
            return -1;
        resident[dev] = per_sm * n_sm;
    }
    static_assert(TX == 32, "classify_kernel works on 32-wide strips");
    const int gx = (a.nx + TX - 1) / TX;
    if (a.mb_ok || (a.tw_prev && a.stage == 2)) {  // from the input's mass bits, or the flags of the stage before
        const int gy = (a.ny + TY - 1) / TY;
        if (launch_after(classify_flags_kernel<T, TY>, dim3((gx * gy + kFlagThreads - 1) / kFlagThreads),
                         dim3(kFlagThreads), 0, st, a, gx, gy) != cudaSuccess)
            return -1;
    } else {
        if (launch_after(classify_kernel<T, TY>, dim3(gx, (a.ny + kStripRows - 1) / kStripRows), dim3(32 * kStripWarps),
                         0, st, a) != cudaSuccess)
            return -1;
    }
    if (launch_after(stage_kernel_list<T, TX, TY, REC, KM, P2>, dim3(resident[dev]), dim3(NTH), smem, st, a, gx) !=
        cudaSuccess)
        return -1;
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}

// the launches that test each tile inside the stage kernel keep no mass bits
template <typename T>
void no_mass_bits(StageArgs<T> &a)
{
    a.mb_in = nullptr;
    a.mb_out = nullptr;
    a.mb_n = nullptr;
    a.mb_ok = 0;
}

// tile 0: 32 x 8 cells (256 threads); tile 1: 32 x 4; tile 2: 32 x 16; tile 3:
// 32 x 4 with two threads per cell on the listed tiles (the launches that test
// each tile themselves take it as 32 x 4)
template <typename T>
int launch_stage_impl(const StageArgs<T> &a_in, int tile, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (a_in.ph.k_mode == 1) {  // the earth-pressure form: the paper's scheme, every tile shape
        if (a_in.wl && !a_in.debug_stage) {
            switch (tile) {
            case 1: return launch_tile_list<T, 32, 4, false, true>(a_in, st);
            case 2: return launch_tile_list<T, 32, 16, false, true>(a_in, st);
            case 3: return launch_tile_list<T, 32, 4, false, true, true>(a_in, st);
            default: return launch_tile_list<T, 32, 8, false, true>(a_in, st);
            }
        }
        StageArgs<T> a = a_in;
        a.wl = nullptr;
        a.wl_n = nullptr;
        no_mass_bits(a);
        switch (tile) {
        case 1:
        case 3: return launch_tile<T, 32, 4, false, false, false, false, true>(a, st);
        case 2: return launch_tile<T, 32, 16, false, false, false, false, true>(a, st);
        default: return launch_tile<T, 32, 8, false, false, false, false, true>(a, st);
        }
    }
    // the model options (viscous term, central-upwind flux, WENO): one tile shape
    const bool vis = a_in.ph.nu_f > 0.0, cu = a_in.ph.scheme == 1, weno = a_in.ph.recon == 1;
    if (a_in.wl && !vis && !cu && !weno && !a_in.debug_stage) {
        switch (tile) {
        case 1: return launch_tile_list<T, 32, 4>(a_in, st);
        case 2: return launch_tile_list<T, 32, 16>(a_in, st);
        case 3: return launch_tile_list<T, 32, 4, false, false, true>(a_in, st);
        default: return launch_tile_list<T, 32, 8>(a_in, st);
        }
    }
    StageArgs<T> a = a_in;  // every tile tests itself
    a.wl = nullptr;
    a.wl_n = nullptr;
    no_mass_bits(a);
    if (weno) {
        if (cu)
            return vis ? launch_tile<T, 32, 8, false, true, true, true>(a, st)
                       : launch_tile<T, 32, 8, false, false, true, true>(a, st);
        return vis ? launch_tile<T, 32, 8, false, true, false, true>(a, st)
                   : launch_tile<T, 32, 8, false, false, false, true>(a, st);
    }
    if (cu)
        return vis ? launch_tile<T, 32, 8, false, true, true>(a, st) : launch_tile<T, 32, 8, false, false, true>(a, st);
    if (vis) return launch_tile<T, 32, 8, false, true>(a, st);
    switch (tile) {
    case 1:
    case 3: return launch_tile<T, 32, 4>(a, st);
    case 2: return launch_tile<T, 32, 16>(a, st);
    default: return launch_tile<T, 32, 8>(a, st);
    }
}

template <typename T>
int launch_stage_rec_impl(const StageArgs<T> &a, void *stream)
{
    if (!a.rec) return -1;
    if (a.ph.k_mode == 1) {
        if (a.wl) return launch_tile_list<T, 32, 8, true, true>(a, (cudaStream_t)stream);
        return launch_tile<T, 32, 8, true, false, false, false, true>(a, (cudaStream_t)stream);
    }
    if (a.wl) return launch_tile_list<T, 32, 8, true>(a, (cudaStream_t)stream);
    return launch_tile<T, 32, 8, true>(a, (cudaStream_t)stream);
}

// The ensemble launch with 32 x TY tiles: the grid is every CTA that fits at
// once (a cooperative launch, so that all of them are resident and can meet);
// with r.nstages == 0 it only reports that grid.
template <typename T, int TY>
int launch_batch_tile(const BatchRun<T> &r, int *grid_out, cudaStream_t st)
{
    constexpr size_t ss = stage_smem_bytes<T, 32, TY>();
    constexpr size_t smem = ss > sizeof(ClassifySmem<T>) ? ss : sizeof(ClassifySmem<T>);
    static int resident[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return -1;
    if (!resident[dev]) {
        int per_sm = 0, n_sm = 0;
        if (cudaFuncSetAttribute(batch_persistent_kernel<T, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel<T, TY>, 32 * TY, smem) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1 || n_sm < 1)
            return -1;
        resident[dev] = per_sm * n_sm;
    }
    if (grid_out) *grid_out = resident[dev];
    if (r.nstages <= 0) return 0;
    BatchRun<T> rr = r;
    void *params[] = {(void *)&rr};
    return cudaLaunchCooperativeKernel((const void *)batch_persistent_kernel<T, TY>, dim3(resident[dev]), dim3(32 * TY),
                                       params, smem, st) == cudaSuccess
               ? 0
               : -1;
}

template <typename T>
int launch_batch_impl(const BatchRun<T> &r, int ty, int *grid_out, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    switch (ty) {
    case 4: return launch_batch_tile<T, 4>(r, grid_out, st);
    case 16: return launch_batch_tile<T, 16>(r, grid_out, st);
    default: return launch_batch_tile<T, 8>(r, grid_out, st);
    }
}

}  // namespace
}  // namespace moses

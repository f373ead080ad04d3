// adjoint.cu -- gradient of a deposit misfit through many steps of the
// two-phase scheme (moses_adjoint_misfit): forward run with the CFL time steps
// and start times recorded and the state checkpointed every C steps, then for
// each segment, from the last to the first, the segment is recomputed with the
// recorded times by the recording stage kernel (keeping U^n, the Heun
// intermediate U* and each stage's record) and swept backwards with the stage
// adjoints of adjoint.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <vector>

#include "adjoint.cuh"
#include "internal.cuh"

using namespace moses;

namespace {

constexpr int ATX = 32, ATY = 8;

// a box of 32 x 8 tiles, inclusive; empty where x1 < x0
struct TileBox {
    int x0, y0, x1, y1;
    bool empty() const { return x1 < x0 || y1 < y0; }
};
inline TileBox box_union(const TileBox &a, const TileBox &b)
{
    if (a.empty()) return b;
    if (b.empty()) return a;
    return TileBox{std::min(a.x0, b.x0), std::min(a.y0, b.y0), std::max(a.x1, b.x1), std::max(a.y1, b.y1)};
}
inline dim3 box_grid(const TileBox &b) { return dim3(b.x1 - b.x0 + 1, b.y1 - b.y0 + 1); }

template <typename T, bool KM>
int launch_adj_face(const AdjArgs<T> &q, cudaStream_t st, const TileBox &box)
{
    static bool attr[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    constexpr size_t smB = FaceAdjSmem<T, ATX, ATY, KM>::bytes;
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        // the largest shared-memory carve-out, so that three FP32 CTAs fit on an SM
        if (cudaFuncSetAttribute(adj_face_kernel<T, ATX, ATY, KM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smB) != cudaSuccess ||
            cudaFuncSetAttribute(adj_face_kernel<T, ATX, ATY, KM>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            return -1;
        attr[dev] = true;
    }
    return launch_after(adj_face_kernel<T, ATX, ATY, KM>, box_grid(box), dim3(ATX * ATY), smB, st, q) == cudaSuccess
               ? 0
               : -1;
}

// the cell kernel on the tiles of `cell`, the face kernel on those of `face`
// (every tile outside them is one that the kernels would leave at once)
template <typename T>
int launch_adj_stage(const AdjArgs<T> &q_in, cudaStream_t st, const TileBox &cell, const TileBox &face)
{
    AdjArgs<T> q = q_in;
    if (!cell.empty()) {
        q.bx0 = cell.x0;
        q.by0 = cell.y0;
        if (launch_after(adj_cell_kernel<T>, box_grid(cell), dim3(256), 0, st, q) != cudaSuccess) return -1;
    }
    if (!face.empty()) {
        q.bx0 = face.x0;
        q.by0 = face.y0;
        if ((q.f.ph.k_mode == 1 ? launch_adj_face<T, true>(q, st, face) : launch_adj_face<T, false>(q, st, face)) != 0)
            return -1;
    }
    if (!q.fold_inline) {
        const int nfold = 6 * (2 * q.f.nx + 2 * q.f.ny);
        if (launch_after(adj_fold_kernel<T>, dim3((nfold + 255) / 256), dim3(256), 0, st, q) != cudaSuccess) return -1;
    }
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -1;
}


// n empty boxes (x min, y min = INT_MAX; x max, y max = -1), widened by the
// classification (StageArgs::wbox)
__global__ void box_init_kernel(int *box, int n)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        box[4 * k] = INT_MAX;
        box[4 * k + 1] = INT_MAX;
        box[4 * k + 2] = -1;
        box[4 * k + 3] = -1;
    }
}

// L = sum (h^s - h^s_target)^2 dx dy with h^s = U1 / J; lam = dL/dU (U1 only)
template <typename T>
__global__ void misfit_kernel(const T *U, const T *R, const T *geo, const double *target, int nx, int ny, int pitch,
                              long long plane, double area, T *lam, double *loss)
{
    const long long n = (long long)nx * ny;
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / nx), i = (int)(e - (long long)j * nx);
        const long long g = cell_index(i, j, pitch);
        const double J = (double)geo[GC_J * plane + g];
        double U1 = (double)U[g];
        if (R) U1 += (double)R[g];
        const double d = U1 / J - target[e];
        acc += d * d * area;
        lam[g] = (T)(2.0 * area * d / J);
#pragma unroll
        for (int c = 1; c < 6; c++) lam[c * plane + g] = T(0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// dL/dh of the release h (U1 = J h phi, U4 = J h (1 - phi), momenta = U v)
template <typename T>
__global__ void release_grad_kernel(const T *lam, const T *U0, const T *geo, const double *phi, int nx, int ny,
                                    int pitch, long long plane, double *out)
{
    const long long n = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / nx), i = (int)(e - (long long)j * nx);
        const long long g = cell_index(i, j, pitch);
        const double J = (double)geo[GC_J * plane + g];
        const double u1 = (double)U0[g], u4 = (double)U0[3 * plane + g];
        double ph = phi ? phi[e] : ((u1 + u4) > 0.0 ? u1 / (u1 + u4) : 0.5);
        double gs = (double)lam[g], gf = (double)lam[3 * plane + g];
        if (u1 > 0.0) gs += ((double)U0[plane + g] * (double)lam[plane + g] + (double)U0[2 * plane + g] * (double)lam[2 * plane + g]) / u1;
        if (u4 > 0.0) gf += ((double)U0[4 * plane + g] * (double)lam[4 * plane + g] + (double)U0[5 * plane + g] * (double)lam[5 * plane + g]) / u4;
        out[e] = J * (ph * gs + (1.0 - ph) * gf);
    }
}

template <typename T>
__global__ void pack_lam_kernel(const T *lam, double *dst, int nx, int ny, int pitch, long long plane)
{
    const long long n = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 6 * n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        const long long r = e - c * n;
        const int j = (int)(r / nx), i = (int)(r - (long long)j * nx);
        dst[e] = (double)lam[c * plane + cell_index(i, j, pitch)];
    }
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

// Partial derivatives of the Savage-Hutter coefficients (reading R10) with
// respect to phi_int ([0]) and delta_b ([1]), in 1/rad; 0 for k_mode 0.  With
// c = cos(phi_int), e = cos(delta_b), r = sqrt(1 - c^2 / e^2) and
// K = 2 (1 -/+ r) / c^2 - 1:
//   dK/dphi   = sin(phi) (4 (1 -/+ r) / c^3 -/+ 2 / (c e^2 r)),
//   dK/ddelta = +/- 2 sin(delta) / (e^3 r)   (K_act: +, K_pass: -).
void earth_pressure_partials(const moses_params &p, double dKa[2], double dKp[2])
{
    dKa[0] = dKa[1] = dKp[0] = dKp[1] = 0.0;
    if (p.k_mode != 1) return;
    const double ph = p.phi_int_deg * M_PI / 180.0, de = p.delta_b_deg * M_PI / 180.0;
    const double c = cos(ph), e = cos(de);
    const double r = sqrt(1.0 - c * c / (e * e));
    dKa[0] = sin(ph) * (4.0 * (1.0 - r) / (c * c * c) - 2.0 / (c * e * e * r));
    dKp[0] = sin(ph) * (4.0 * (1.0 + r) / (c * c * c) + 2.0 / (c * e * e * r));
    dKa[1] = 2.0 * sin(de) / (e * e * e * r);
    dKp[1] = -dKa[1];
}

template <typename T>
int adjoint_impl(moses_sim *s, int nsteps, int C, const double *hs_target, double *loss_out, double *g_params,
                 double *g_state0, double *g_release_h, const double *release_phi, double *timing)
{
    cudaStream_t st = s->stream;
    const int nx = s->nx, ny = s->ny, pitch = s->pitch;
    const long long plane = s->plane;
    const long long n = (long long)nx * ny;
    const size_t sb = (s->prec == MOSES_FP32 ? 8 : 6) * (size_t)plane * sizeof(T);  // a full state buffer
    const size_t lb = 6 * (size_t)plane * sizeof(T);
    const int nck = (nsteps + C - 1) / C;
    const size_t rb = 6 * (size_t)plane * sizeof(T);  // one stage's record
    DevBuf dts_d, ck, seg, recb, lam, lamA, lpre, ldp, gpar, loss_d, tgt, phi_d, hbuf, zkseg, twseg, lamz, mbseg, boxd;
    // tiles of the 32 x 8 launches (the forward run, the recording recompute
    // and the adjoint kernels share this tiling)
    const int tgx = (nx + 31) / 32, tgy = (ny + 7) / 8;
    const size_t nt = (size_t)tgx * tgy;
    CK(cudaMalloc(&dts_d.p, 2 * sizeof(double) * nsteps));
    CK(cudaMalloc(&ck.p, sb * nck));
    // two sets of segment buffers: the recompute of one segment runs on a
    // second stream while the reverse sweep of the segment after it runs
    CK(cudaMalloc(&seg.p, 2 * sb * (2 * C + 1)));
    CK(cudaMalloc(&recb.p, 2 * rb * 2 * C));
    for (DevBuf *b : {&lam, &lamA, &lpre}) {
        CK(cudaMalloc(&b->p, lb));
        CK(cudaMemsetAsync(b->p, 0, lb, st));
    }
    CK(cudaMalloc(&ldp.p, 2 * (size_t)plane * sizeof(T)));
    CK(cudaMemsetAsync(ldp.p, 0, 2 * (size_t)plane * sizeof(T), st));
    CK(cudaMalloc(&gpar.p, 4 * sizeof(double)));
    CK(cudaMemsetAsync(gpar.p, 0, 4 * sizeof(double), st));
    CK(cudaMalloc(&loss_d.p, sizeof(double)));
    CK(cudaMemsetAsync(loss_d.p, 0, sizeof(double), st));
    // per set: known-zero tile flags of the recompute's output buffers
    // (segU(1..C), segS(0..C-1); each with its record buffer, a fixed pairing
    // across segments) and the stages' tile-wet maps of a segment; the
    // per-tile flags of lam's momentum adjoints (all 0 after the misfit)
    CK(cudaMalloc(&zkseg.p, 2 * nt * (2 * C + 1)));
    CK(cudaMemsetAsync(zkseg.p, 0, 2 * nt * (2 * C + 1), st));
    CK(cudaMalloc(&twseg.p, 2 * nt * 2 * C));
    // mass bits of each buffer of the two segment sets (written before read)
    CK(cudaMalloc(&mbseg.p, 2 * sizeof(unsigned short) * nt * (2 * C + 1)));
    CK(cudaMemsetAsync(twseg.p, 0, 2 * nt * 2 * C, st));
    CK(cudaMalloc(&lamz.p, nt));
    CK(cudaMemsetAsync(lamz.p, 1, nt, st));
    // per set and stage of a segment: the box of the tiles the recompute's
    // classification listed, read back by the host before the segment's sweep
    CK(cudaMalloc(&boxd.p, sizeof(int) * 4 * 2 * 2 * C));
    struct PinnedInts {
        int *p = nullptr;
        ~PinnedInts() { cudaFreeHost(p); }
    } boxh;
    CK(cudaMallocHost(&boxh.p, sizeof(int) * 4 * 2 * 2 * C));
    CK(cudaMalloc(&tgt.p, sizeof(double) * n));
    CK(cudaMemcpyAsync(tgt.p, hs_target, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    if (release_phi) {
        CK(cudaMalloc(&phi_d.p, sizeof(double) * n));
        CK(cudaMemcpyAsync(phi_d.p, release_phi, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    }
    char *ckp = (char *)ck.p;
    // set b of the segment buffers
    auto segU = [&](int b, int q) { return (T *)((char *)seg.p + sb * ((2 * C + 1) * b + q)); };  // U^{start+q}
    auto segS = [&](int b, int q) { return (T *)((char *)seg.p + sb * ((2 * C + 1) * b + C + 1 + q)); };  // U*
    auto rec = [&](int b, int q, int stage) { return (T *)((char *)recb.p + rb * (2 * C * b + 2 * q + stage - 1)); };
    auto zks = [&](int b) { return (unsigned char *)zkseg.p + nt * (2 * C + 1) * b; };
    auto tws = [&](int b) { return (unsigned char *)twseg.p + nt * 2 * C * b; };
    // mass bits of segU(b, m) at m, of segS(b, m) at C + 1 + m
    auto mbs = [&](int b) { return (unsigned short *)mbseg.p + nt * (2 * C + 1) * b; };
    // the listed-tile box of stage (m, stage) of set b
    auto boxes = [&](int b) { return (int *)boxd.p + 4 * 2 * C * b; };

    cudaEvent_t ev[4];
    for (int q = 0; q < 4; q++) CK(cudaEventCreate(&ev[q]));
    CK(cudaEventRecord(ev[0], st));

    // ---- forward run, CFL time steps recorded, checkpoints every C steps ----
    StageArgs<T> a1 = base_args<T>(s), a2 = base_args<T>(s);
    a1.Uin = (const T *)s->U;
    a1.Uout = (T *)s->Us;
    a1.Rin = rem<T>(s, s->U);
    a1.Rout = rem<T>(s, s->Us);
    a1.stage = 1;
    a2.Uin = (const T *)s->Us;
    a2.Un = (const T *)s->U;
    a2.Uout = (T *)s->U;
    a2.Rin = rem<T>(s, s->Us);
    a2.Rn = rem<T>(s, s->U);
    a2.Rout = rem<T>(s, s->U);
    a2.stage = 2;
    a2.want_amax = 1;
    // the forward run steps as moses_step does (wet-tile list, known-zero tile
    // flags of U and U* for the 32 x 8 tiling, cleared first)
    a1.wl = a2.wl = s->wl;
    a1.wl_n = a2.wl_n = s->wl_n;
    a1.tw_next = s->tw[0];
    a2.tw_prev = s->tw[0];
    a2.tw_next = s->tw[1];
    CK(cudaMemsetAsync(s->zk, 0, 2 * nt, st));
    a1.zk = s->zk + nt;
    a2.zk = s->zk;
    // mass bits of U and U* (the first stage of the first step classifies
    // from the data and writes U's)
    a1.mb_in = s->mb;
    a1.mb_out = s->mb + nt;
    a2.mb_in = s->mb + nt;
    a2.mb_n = s->mb;
    a2.mb_out = s->mb;
    a2.mb_ok = 1;
    const double zero = 0.0;
    CK(cudaMemcpyAsync(&s->ctl->dt_fixed, &zero, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(&s->ctl->t_end, &zero, sizeof(double), cudaMemcpyHostToDevice, st));
    // the first stage of each step logs its start time and time step
    a1.t_log = (double *)dts_d.p + nsteps;
    a1.dt_log = (double *)dts_d.p;
    for (int k = 0; k < nsteps; k++) {
        if (k % C == 0) CK(cudaMemcpyAsync(ckp + sb * (k / C), s->U, sb, cudaMemcpyDeviceToDevice, st));
        a1.log_idx = k;
        a1.mb_ok = k > 0;
        if (launch_stage<T>(a1, 0, st) || launch_stage<T>(a2, 0, st)) return fail(s, MOSES_ECUDA, "forward launch");
    }
    CK(cudaGetLastError());
    Ctl ctl_end;
    CK(cudaMemcpyAsync(&ctl_end, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    misfit_kernel<T><<<grid_for(n), 256, 0, st>>>((const T *)s->U, rem<T>(s, s->U), (const T *)s->geo,
                                                   (const double *)tgt.p, nx, ny, pitch, plane, s->dx * s->dy,
                                                   (T *)lam.p, (double *)loss_d.p);
    std::vector<double> dts(2 * (size_t)nsteps);  // time steps, then start times
    CK(cudaMemcpyAsync(dts.data(), dts_d.p, 2 * sizeof(double) * nsteps, cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(ev[1], st));
    CK(cudaStreamSynchronize(st));

    // ---- backward over the segments ----
    AdjArgs<T> q{};
    q.lam_pre = (T *)lpre.p;
    q.lam_dp = (T *)ldp.p;
    q.g_param = (double *)gpar.p;
    q.lam_next = (const T *)lam.p;
    q.tgx = tgx;
    q.tgy = tgy;
    q.lamz = (unsigned char *)lamz.p;
    // every ghost's source lies in the tile that owns the ghost (32 x 8 tiles)
    q.fold_inline = (nx == 1 || nx % ATX != 1) && (ny == 1 || ny % ATY != 1);
    // The recompute of segment k runs on stream rs into set k & 1, after the
    // sweep that last read that set (segment k + 2); the sweep of segment k
    // runs on st after its recompute.  Issuing the recompute of k - 1 before
    // the sweep of k lets the two overlap: both are latency-bound on a few
    // wet tiles.  Only the recompute touches the control block and the
    // wet-tile list; the sweep reads its set and its own adjoint buffers.
    cudaStream_t rs = nullptr;
    cudaEvent_t rec_done[2] = {nullptr, nullptr}, sweep_done[2] = {nullptr, nullptr};
    struct Streams {
        cudaStream_t &rs;
        cudaEvent_t *a, *b;
        ~Streams()
        {
            if (rs) cudaStreamDestroy(rs);
            for (int k = 0; k < 2; k++) {
                if (a[k]) cudaEventDestroy(a[k]);
                if (b[k]) cudaEventDestroy(b[k]);
            }
        }
    } streams_guard{rs, rec_done, sweep_done};
    CK(cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking));
    for (int k = 0; k < 2; k++) {
        CK(cudaEventCreateWithFlags(&rec_done[k], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&sweep_done[k], cudaEventDisableTiming));
    }
    bool swept[2] = {false, false};
    auto recompute = [&](const int kseg) -> int {
        const int b = kseg & 1, start = kseg * C, end = std::min(start + C, nsteps);
        if (swept[b]) CK(cudaStreamWaitEvent(rs, sweep_done[b], 0));
        CK(cudaMemcpyAsync(segU(b, 0), ckp + sb * kseg, sb, cudaMemcpyDeviceToDevice, rs));
        box_init_kernel<<<1, 256, 0, rs>>>(boxes(b), 2 * C);
        for (int k = start; k < end; k++) {
            const int m = k - start;
            StageArgs<T> r1 = a1, r2 = a2;
            // the step's start time and time step as the forward run took them
            r1.t_log = r1.dt_log = nullptr;
            r1.fix = 1;
            r1.fix_t = dts[nsteps + k];
            r1.fix_dt = dts[k];
            // (the recording stages run on the wet-tile list too, tile 32 x 8)
            r1.Uin = segU(b, m);
            r1.Uout = segS(b, m);
            r1.Rin = rem<T>(s, segU(b, m));
            r1.Rout = rem<T>(s, segS(b, m));
            r1.rec = rec(b, m, 1);
            r2.Uin = segS(b, m);
            r2.Un = segU(b, m);
            r2.Uout = segU(b, m + 1);
            r2.Rin = rem<T>(s, segS(b, m));
            r2.Rn = rem<T>(s, segU(b, m));
            r2.Rout = rem<T>(s, segU(b, m + 1));
            r2.rec = rec(b, m, 2);
            r2.want_amax = 0;
            r1.zk = zks(b) + nt * (C + 1 + m);
            r2.zk = zks(b) + nt * (m + 1);
            r1.tw_next = tws(b) + nt * (2 * m);
            r2.tw_prev = tws(b) + nt * (2 * m);
            r2.tw_next = tws(b) + nt * (2 * m + 1);
            // mass bits: the segment's first stage classifies from the data
            r1.mb_in = mbs(b) + nt * m;
            r1.mb_out = mbs(b) + nt * (C + 1 + m);
            r1.mb_ok = m > 0;
            r2.mb_in = mbs(b) + nt * (C + 1 + m);
            r2.mb_n = mbs(b) + nt * m;
            r2.mb_out = mbs(b) + nt * (m + 1);
            r2.mb_ok = 1;
            r1.wbox = boxes(b) + 4 * (2 * m);
            r2.wbox = boxes(b) + 4 * (2 * m + 1);
            if (launch_stage_rec<T>(r1, rs) || launch_stage_rec<T>(r2, rs))
                return fail(s, MOSES_ECUDA, "recompute launch");
        }
        CK(cudaMemcpyAsync(boxh.p + 4 * 2 * C * b, boxes(b), sizeof(int) * 4 * 2 * C, cudaMemcpyDeviceToHost, rs));
        CK(cudaEventRecord(rec_done[b], rs));
        return MOSES_OK;
    };
    // the near box of a stage: its listed tiles' box widened by the two tiles
    // of the adjoint kernels' far test (AdjArgs::tw), within the grid
    auto near_box = [&](int b, int idx) {
        const int *w = boxh.p + 4 * (2 * C * b + idx);
        if (w[2] < w[0]) return TileBox{0, 0, -1, -1};
        return TileBox{std::max(w[0] - 2, 0), std::max(w[1] - 2, 0), std::min(w[2] + 2, tgx - 1),
                       std::min(w[3] + 2, tgy - 1)};
    };
    // the near box of the last first-stage reverse: its tiles may hold momentum
    // adjoints that the next one zeroes where it finds them far (AdjArgs::lamz)
    TileBox prev1{0, 0, -1, -1};
    auto sweep = [&](const int kseg) -> int {
        const int b = kseg & 1, start = kseg * C, end = std::min(start + C, nsteps);
        CK(cudaStreamWaitEvent(st, rec_done[b], 0));
        CK(cudaEventSynchronize(rec_done[b]));  // the segment's boxes (the sweep before keeps the GPU busy)
        for (int k = end - 1; k >= start; k--) {
            const int m = k - start;
            q.f = base_args<T>(s);
            q.f.debug_stage = 1;
            q.f.dbg_dt = dts[k];
            q.U_next = segU(b, m + 1);
            // stage 2 at U*: lam_out = the Heun term of lam^{n+1} -> lamA
            q.f.Uin = segS(b, m);
            q.f.rec = rec(b, m, 2);
            q.tw = tws(b) + nt * (2 * m + 1);
            q.heun = 2;
            q.lam_out = nullptr;
            q.lam_in = (T *)lamA.p;
            const TileBox n2 = near_box(b, 2 * m + 1), n1 = near_box(b, 2 * m);
            if (launch_adj_stage<T>(q, st, n2, n2)) return fail(s, MOSES_ECUDA, "adjoint launch");
            // stage 1 at U^n: lam_out = lamA; lam^n = its input adjoint + the Heun term, over lam^{n+1}
            q.f.Uin = segU(b, m);
            q.f.rec = rec(b, m, 1);
            q.tw = tws(b) + nt * (2 * m);
            q.heun = 1;
            q.lam_out = (const T *)lamA.p;
            q.lam_in = (T *)lam.p;
            if (launch_adj_stage<T>(q, st, box_union(n1, prev1), n1)) return fail(s, MOSES_ECUDA, "adjoint launch");
            prev1 = n1;
        }
        CK(cudaEventRecord(sweep_done[b], st));
        swept[b] = true;
        return MOSES_OK;
    };
    // the recompute stream starts after the forward run and the misfit
    CK(cudaEventRecord(sweep_done[0], st));
    CK(cudaStreamWaitEvent(rs, sweep_done[0], 0));
    int rc = recompute(nck - 1);
    for (int kseg = nck - 1; kseg >= 0 && rc == 0; kseg--) {
        if (kseg > 0) rc = recompute(kseg - 1);
        if (rc == 0) rc = sweep(kseg);
    }
    if (rc) return rc;
    CK(cudaGetLastError());
    CK(cudaEventRecord(ev[2], st));
    // ---- outputs; the state and the clock go back to the end of the forward run ----
    double gp[4] = {0, 0, 0, 0}, loss = 0;
    CK(cudaMemcpyAsync(gp, gpar.p, sizeof(gp), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&loss, loss_d.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (g_state0) {
        CK(cudaMalloc(&hbuf.p, sizeof(double) * 6 * n));
        pack_lam_kernel<T><<<grid_for(6 * n), 256, 0, st>>>((const T *)lam.p, (double *)hbuf.p, nx, ny, pitch, plane);
        CK(cudaMemcpyAsync(g_state0, hbuf.p, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, st));
    }
    if (g_release_h) {
        DevBuf gh;
        CK(cudaMalloc(&gh.p, sizeof(double) * n));
        release_grad_kernel<T><<<grid_for(n), 256, 0, st>>>((const T *)lam.p, (const T *)ckp, (const T *)s->geo,
                                                            (const double *)phi_d.p, nx, ny, pitch, plane,
                                                            (double *)gh.p);
        CK(cudaMemcpyAsync(g_release_h, gh.p, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    CK(cudaMemcpyAsync(s->ctl, &ctl_end, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(ev[3], st));
    CK(cudaStreamSynchronize(st));
    if (timing) {
        float f = 0, b = 0;
        cudaEventElapsedTime(&f, ev[0], ev[1]);
        cudaEventElapsedTime(&b, ev[1], ev[2]);
        timing[0] = f;
        timing[1] = b;
    }
    for (int q2 = 0; q2 < 4; q2++) cudaEventDestroy(ev[q2]);
    const double tand = s->ph.tan_delta;
    if (loss_out) *loss_out = loss;
    if (g_params) {
        // delta_b acts through tan(delta_b) and, with k_mode 1, through
        // K_act and K_pass; phi_int only through them (k_mode 0: not at all)
        double dKa[2], dKp[2];
        earth_pressure_partials(s->p, dKa, dKp);
        g_params[0] = (gp[0] * (1.0 + tand * tand) + gp[2] * dKa[1] + gp[3] * dKp[1]) * (M_PI / 180.0);
        g_params[1] = (gp[2] * dKa[0] + gp[3] * dKp[0]) * (M_PI / 180.0);  // per degree of phi_int
        g_params[2] = gp[1];
    }
    return MOSES_OK;
}

}  // namespace

int moses_adjoint_misfit(moses_sim *s, int nsteps, int ckpt_every, const double *hs_target, double *loss,
                         double g_params[3], double *g_state0, double *g_release_h, const double *release_phi,
                         double timing_ms[2])
{
    const ZkReset zr{s};
    if (!s) return MOSES_EINVAL;
    if (!hs_target) return fail(s, MOSES_EINVAL, "hs_target must be non-NULL");
    if (nsteps < 1) return fail(s, MOSES_EINVAL, "nsteps must be >= 1");
    if (ckpt_every < 1) ckpt_every = (int)std::ceil(std::sqrt((double)nsteps));
    if (ckpt_every > nsteps) ckpt_every = nsteps;
    if (s->p.nu_f != 0.0) return fail(s, MOSES_EINVAL, "the adjoint does not cover the viscous term");
    if (s->p.scheme != MOSES_SCHEME_CENTRAL || s->ph.recon != 0 || s->ph.rk != 2)
        return fail(s, MOSES_EINVAL, "the adjoint covers the paper's scheme only (central, minmod, two-step)");
    if (s->ph.k_mode == 1 && !(s->p.delta_b_deg < s->p.phi_int_deg))
        return fail(s, MOSES_EINVAL, "the adjoint of k_mode 1 needs delta_b < phi_int (K has no derivative at equality)");
    if (is_strip(s)) return fail(s, MOSES_EINVAL, "the adjoint covers a whole domain, not a strip of one");
    if (!s->have_state) return fail(s, MOSES_ESTATE, "no state");
    return s->prec == MOSES_FP64
               ? adjoint_impl<double>(s, nsteps, ckpt_every, hs_target, loss, g_params, g_state0, g_release_h,
                                      release_phi, timing_ms)
               : adjoint_impl<float>(s, nsteps, ckpt_every, hs_target, loss, g_params, g_state0, g_release_h,
                                     release_phi, timing_ms);
}

namespace {
template <typename T>
__global__ void unpack_lam_kernel(const double *src, T *lam, int nx, int ny, int pitch, long long plane)
{
    const long long n = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 6 * n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        const long long r = e - c * n;
        const int j = (int)(r / nx), i = (int)(r - (long long)j * nx);
        lam[c * plane + cell_index(i, j, pitch)] = (T)src[e];
    }
}

template <typename T>
int stage_adjoint_impl(moses_sim *s, double t, double dt, const double *lam_out, double *lam_in, double *g_param)
{
    cudaStream_t st = s->stream;
    const long long n = (long long)s->nx * s->ny;
    const size_t lb = 6 * (size_t)s->plane * sizeof(T);
    DevBuf lo, li, lpre, ldp, gp, hb, recb;
    CK(cudaMalloc(&recb.p, lb));
    CK(cudaMalloc(&lo.p, lb));
    CK(cudaMalloc(&li.p, lb));
    CK(cudaMalloc(&lpre.p, lb));
    CK(cudaMalloc(&ldp.p, 2 * (size_t)s->plane * sizeof(T)));
    CK(cudaMalloc(&gp.p, 4 * sizeof(double)));
    CK(cudaMalloc(&hb.p, sizeof(double) * 6 * n));
    CK(cudaMemsetAsync(lo.p, 0, lb, st));
    CK(cudaMemsetAsync(li.p, 0, lb, st));
    CK(cudaMemsetAsync(gp.p, 0, 4 * sizeof(double), st));
    CK(cudaMemcpyAsync(hb.p, lam_out, sizeof(double) * 6 * n, cudaMemcpyHostToDevice, st));
    unpack_lam_kernel<T><<<grid_for(6 * n), 256, 0, st>>>((const double *)hb.p, (T *)lo.p, s->nx, s->ny, s->pitch,
                                                          s->plane);
    // the stage again, recording what the cell adjoint needs (ghosts of U are
    // those of time t, filled by moses_stage)
    StageArgs<T> f = base_args<T>(s);
    f.Uin = (const T *)s->U;
    f.Uout = (T *)s->Us;
    f.Rin = rem<T>(s, s->U);
    f.Rout = rem<T>(s, s->Us);
    f.stage = 1;
    f.debug_stage = 1;
    f.dbg_t = t;
    f.dbg_dt = dt;
    f.rec = (T *)recb.p;
    if (launch_stage_rec<T>(f, st)) return fail(s, MOSES_ECUDA, "recording stage launch");
    AdjArgs<T> q{};
    q.f = f;
    q.lam_out = (const T *)lo.p;
    q.lam_in = (T *)li.p;
    q.lam_pre = (T *)lpre.p;
    q.lam_dp = (T *)ldp.p;
    q.g_param = (double *)gp.p;
    const TileBox all{0, 0, (s->nx + ATX - 1) / ATX - 1, (s->ny + ATY - 1) / ATY - 1};
    if (launch_adj_stage<T>(q, st, all, all)) return fail(s, MOSES_ECUDA, "adjoint launch");
    pack_lam_kernel<T><<<grid_for(6 * n), 256, 0, st>>>((const T *)li.p, (double *)hb.p, s->nx, s->ny, s->pitch,
                                                        s->plane);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(lam_in, hb.p, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, st));
    double g[4];
    CK(cudaMemcpyAsync(g, gp.p, sizeof(g), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (g_param) {
        // tan(delta_b) also moves K_act and K_pass: d delta_b / d tan = cos^2
        double dKa[2], dKp[2];
        earth_pressure_partials(s->p, dKa, dKp);
        const double c2 = 1.0 / (1.0 + s->ph.tan_delta * s->ph.tan_delta);
        g_param[0] = g[0] + (g[2] * dKa[1] + g[3] * dKp[1]) * c2;
        g_param[1] = g[1];
        g_param[2] = g[2] * dKa[0] + g[3] * dKp[0];  // per radian of phi_int
    }
    return MOSES_OK;
}
}  // namespace

int moses_stage_adjoint(moses_sim *s, double t, double dt, const double *lam_out, double *lam_in, double *g_param)
{
    const ZkReset zr{s};
    if (!s || !lam_out || !lam_in) return MOSES_EINVAL;
    if (!(std::isfinite(dt) && dt >= 0)) return fail(s, MOSES_EINVAL, "bad dt");
    if (s->p.nu_f != 0.0 || s->p.scheme != MOSES_SCHEME_CENTRAL || s->ph.recon != 0 || s->ph.rk != 2)
        return fail(s, MOSES_EINVAL, "the adjoint covers the paper's scheme without the viscous term");
    if (s->ph.k_mode == 1 && !(s->p.delta_b_deg < s->p.phi_int_deg))
        return fail(s, MOSES_EINVAL, "the adjoint of k_mode 1 needs delta_b < phi_int (K has no derivative at equality)");
    // ghosts of the current state at time t, as moses_stage sees them
    double *tmp = nullptr;
    CK(cudaMallocHost(&tmp, sizeof(double) * 6 * (size_t)s->nx * s->ny));
    int rc = moses_stage(s, t, dt, tmp);
    cudaFreeHost(tmp);
    if (rc) return rc;
    return s->prec == MOSES_FP64 ? stage_adjoint_impl<double>(s, t, dt, lam_out, lam_in, g_param)
                                 : stage_adjoint_impl<float>(s, t, dt, lam_out, lam_in, g_param);
}

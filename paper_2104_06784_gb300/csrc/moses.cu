// moses.cu -- C-ABI of the two-phase shallow-flow step (include/moses.h):
// simulation object, device memory, the one-time geometry pass (Sect. 2.1,
// App. A: J_b, Omega_b^-1, basal normal and its derivatives), the initial
// ghost fill, the exact CFL max-reduction and the FP64 budget reductions.
// The per-step stage kernels live in stage.cuh (instantiated in
// stage_f64.cu / stage_f32.cu through stage_launch.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/moses.h"
#include "moses_dev.cuh"
#include "batch.cuh"
#include "stage.cuh"

using namespace moses;

#include "internal.cuh"

std::string g_create_err;

// ---------------------------------------------------------------------------
// geometry pass (once per DEM)

// DEM value after extrapolating linearly in X over rows 0..ny-1 (3 layers)
__device__ __forceinline__ double dem_x(const double *dem, int nx, int i, int j)
{
    if (i >= 0 && i < nx) return dem[(long long)j * nx + i];
    if (i < 0) {
        const double b0 = dem[(long long)j * nx], b1 = nx > 1 ? dem[(long long)j * nx + 1] : b0;
        return b0 + (double)(-i) * (b0 - b1);
    }
    const double e0 = dem[(long long)j * nx + nx - 1], e1 = nx > 1 ? dem[(long long)j * nx + nx - 2] : e0;
    return e0 + (double)(i - nx + 1) * (e0 - e1);
}

// then in Y over all (extended) columns
__device__ __forceinline__ double dem_xy(const double *dem, int nx, int ny, int i, int j)
{
    if (j >= 0 && j < ny) return dem_x(dem, nx, i, j);
    if (j < 0) {
        const double b0 = dem_x(dem, nx, i, 0), b1 = ny > 1 ? dem_x(dem, nx, i, 1) : b0;
        return b0 + (double)(-j) * (b0 - b1);
    }
    const double e0 = dem_x(dem, nx, i, ny - 1), e1 = ny > 1 ? dem_x(dem, nx, i, ny - 2) : e0;
    return e0 + (double)(j - ny + 1) * (e0 - e1);
}

__global__ void extend_dem_kernel(const double *dem, int nx, int ny, double *bext)
{
    const int W = nx + 6, H = ny + 6;
    const long long n = (long long)W * H;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int jj = (int)(e / W), ii = (int)(e - (long long)jj * W);
        bext[e] = dem_xy(dem, nx, ny, ii - 3, jj - 3);
    }
}

struct Slopes {
    double bX, bY;
};

template <typename T>
__global__ void geometry_kernel(const double *bext, int nx, int ny, int pitch, long long plane, double dx,
                                double dy, Phys ph, T *geo, int with_slopes)
{
    const int W = nx + 4, H = ny + 4;  // padded cell range [-2, n+2)
    const long long n = (long long)W * H;
    const int BW = nx + 6;
    auto B = [&](int i, int j) { return bext[(long long)(j + 3) * BW + (i + 3)]; };
    auto slopes = [&](int i, int j) {
        return Slopes{(B(i + 1, j) - B(i - 1, j)) / (2.0 * dx), (B(i, j + 1) - B(i, j - 1)) / (2.0 * dy)};
    };
    auto put = [&](int q, long long g, double v) { geo[q * plane + g] = (T)v; };
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / W) - 2, i = (int)(e % W) - 2;
        const long long g = cell_index(i, j, pitch);
        // cell centre: slopes by central differences, curvature by second
        // differences; Omega_b = [(1,0,bX), (0,1,bY), n], J = det, A = 2x2
        // block of its inverse (the inverse metric of the bed surface)
        {
            const Slopes s = slopes(i, j);
            const double bXX = (B(i + 1, j) - 2.0 * B(i, j) + B(i - 1, j)) / (dx * dx);
            const double bYY = (B(i, j + 1) - 2.0 * B(i, j) + B(i, j - 1)) / (dy * dy);
            const double bXY = (B(i + 1, j + 1) - B(i + 1, j - 1) - B(i - 1, j + 1) + B(i - 1, j - 1)) / (4.0 * dx * dy);
            const double s2 = 1.0 + (s.bX * s.bX + s.bY * s.bY);
            const double J = sqrt(s2), c = 1.0 / J, c2 = 1.0 / s2;
            const double A11 = (1.0 + s.bY * s.bY) * c2, A12 = -s.bX * s.bY * c2, A22 = (1.0 + s.bX * s.bX) * c2;
            put(GC_J, g, J);
            put(GC_C, g, c);
            put(GC_JHD, g, J * ph.h_dry);
            put(GC_GC1, g, ph.g_1ma * c);
            put(GC_GCF, g, ph.g * c);
            put(GC_BX, g, s.bX);
            put(GC_BY, g, s.bY);
            put(GC_MNX, g, -c * s.bX);
            put(GC_MNY, g, -c * s.bY);
            put(GC_A11, g, A11);
            put(GC_A12, g, A12);
            put(GC_A22, g, A22);
            put(GC_KXX, g, c * bXX);
            put(GC_KXY2, g, 2.0 * c * bXY);
            put(GC_KYY, g, c * bYY);
            put(GC_SXS, g, ph.kap_s * ph.K_pass * A11 * c2);
            put(GC_SXF, g, 2.0 * ph.kap_f * A11 * c2);
            put(GC_SYS, g, ph.kap_s * ph.K_pass * A22 * c2);
            put(GC_SYF, g, 2.0 * ph.kap_f * A22 * c2);
        }
        // x-face (i+1/2, j): normal slope by the face difference, transverse
        // slope as the mean of the two cells' central differences
        if (i < nx + 1) {
            const double bX = (B(i + 1, j) - B(i, j)) / dx;
            const double bY = 0.5 * (slopes(i, j).bY + slopes(i + 1, j).bY);
            const double s2 = 1.0 + (bX * bX + bY * bY);
            const double c2 = 1.0 / s2;
            const double An = (1.0 + bY * bY) * c2 * c2, At = -bX * bY * c2 * c2;  // A11 c^2, A12 c^2
            put(GX_JHD, g, sqrt(s2) * ph.h_dry);
            put(GX_SN, g, ph.kap_s * An);
            put(GX_ST, g, ph.kap_s * At);
            put(GX_FN, g, ph.kap_f * An);
            put(GX_FT, g, ph.kap_f * At);
            put(GX_FN2, g, 2.0 * ph.kap_f * An);
            put(GX_HG, g, ph.half_g * c2);
        }
        if (j < ny + 1) {
            const double bY = (B(i, j + 1) - B(i, j)) / dy;
            const double bX = 0.5 * (slopes(i, j).bX + slopes(i, j + 1).bX);
            const double s2 = 1.0 + (bX * bX + bY * bY);
            const double c2 = 1.0 / s2;
            const double An = (1.0 + bX * bX) * c2 * c2, At = -bX * bY * c2 * c2;  // A22 c^2, A21 c^2
            put(GY_JHD, g, sqrt(s2) * ph.h_dry);
            put(GY_SN, g, ph.kap_s * An);
            put(GY_ST, g, ph.kap_s * At);
            put(GY_FN, g, ph.kap_f * An);
            put(GY_FT, g, ph.kap_f * At);
            put(GY_FN2, g, 2.0 * ph.kap_f * An);
            put(GY_HG, g, ph.half_g * c2);
        }
        if (with_slopes) {
            const Slopes s = slopes(i, j);
            put(GS_SX, g, s.bX);
            put(GS_SY, g, s.bY);
            if (i < nx + 1) put(GS_DBX, g, (B(i + 1, j) - B(i, j)) / dx);
            if (j < ny + 1) put(GS_DBY, g, (B(i, j + 1) - B(i, j)) / dy);
        }
    }
}

// ---------------------------------------------------------------------------
// state kernels

template <typename T>
__global__ void fill_ghosts_kernel(const StageArgs<T> a, T *U, double tg)
{
    const int nx = a.nx, ny = a.ny;
    const long long n = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / nx), i = (int)(e - (long long)j * nx);
        if (!(i < 2 || i >= nx - 2 || j < 2 || j >= ny - 2)) continue;
        const long long g = cell_index(i, j, a.pitch);
        T v[6];
#pragma unroll
        for (int c = 0; c < 6; c++) v[c] = U[c * a.plane + g];
        write_ghosts(U, a.geo, a, i, j, v, tg);
    }
}

template <typename T>
__global__ void max_speed_kernel(const T *U, const T *geo, int nx, int j0, int j1, int pitch, long long plane,
                                 unsigned long long *out)
{
    const long long n = (long long)nx * (j1 - j0);  // the rows [j0, j1)
    double m = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int j = j0 + (int)(e / nx), i = (int)(e - (long long)(j - j0) * nx);
        const long long g = cell_index(i, j, pitch);
        T u[6];
#pragma unroll
        for (int c = 0; c < 6; c++) u[c] = U[c * plane + g];
        m = fmax(m, (double)cell_speed(u, geo, plane, g));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); q++) m = fmax(m, w[q]);
        atomicMax(out, (unsigned long long)__double_as_longlong(m));
    }
}

// dense doubles [c][j][i] -> padded state of type T (interior only); with R
// (FP32 form) the masses are split into value + rounding remainder
template <typename T>
__global__ void unpack_kernel(const double *src, T *U, T *R, int nx, int ny, int pitch, long long plane)
{
    const long long n = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 6 * n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        const long long r = e - c * n;
        const int j = (int)(r / nx), i = (int)(r - (long long)j * nx);
        const long long g = cell_index(i, j, pitch);
        const double v = src[e];
        const T hi = (T)v;
        U[c * plane + g] = hi;
        if (R && (c == 0 || c == 3)) R[(c / 3) * plane + g] = (T)(v - (double)hi);
    }
}

template <typename T>
__global__ void pack_kernel(const T *U, const T *R, double *dst, int nx, int ny, int pitch, long long plane)
{
    const long long n = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 6 * n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        const long long r = e - c * n;
        const int j = (int)(r / nx), i = (int)(r - (long long)j * nx);
        const long long g = cell_index(i, j, pitch);
        double v = (double)U[c * plane + g];
        if (R && (c == 0 || c == 3)) v += (double)R[(c / 3) * plane + g];
        dst[e] = v;
    }
}

// rows [j0, j0 + nrows) of the state (and, FP32, of the two mass remainder
// planes) <-> a dense buffer [plane][row][i] of doubles (exact both ways for
// values of the simulation's own type)
template <typename T>
__global__ void rows_pack_kernel(const T *U, const T *R, double *dst, int nx, int j0, int nrows, int pitch,
                                 long long plane)
{
    const int np = R ? 8 : 6;
    const long long n = (long long)nx * nrows;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < np * n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        const long long r = e - c * n;
        const int j = j0 + (int)(r / nx), i = (int)(r - (long long)(j - j0) * nx);
        const long long g = cell_index(i, j, pitch);
        dst[e] = c < 6 ? (double)U[c * plane + g] : (double)R[(c - 6) * plane + g];
    }
}

template <typename T>
__global__ void rows_unpack_kernel(const double *src, T *U, T *R, int nx, int j0, int nrows, int pitch, long long plane)
{
    const int np = R ? 8 : 6;
    const long long n = (long long)nx * nrows;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < np * n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        const long long r = e - c * n;
        const int j = j0 + (int)(r / nx), i = (int)(r - (long long)(j - j0) * nx);
        const long long g = cell_index(i, j, pitch);
        if (c < 6) U[c * plane + g] = (T)src[e];
        else R[(c - 6) * plane + g] = (T)src[e];
    }
}

// the ghost cells that the cells of rows [j0, j1) own (write_ghosts), at
// the control block's time: after rows were replaced from outside
template <typename T>
__global__ void fill_ghosts_rows_kernel(const StageArgs<T> a, T *U, int j0, int j1)
{
    const int nx = a.nx, ny = a.ny;
    const long long n = (long long)nx * (j1 - j0);
    const double tg = a.ctl->t;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int j = j0 + (int)(e / nx), i = (int)(e - (long long)(j - j0) * nx);
        if (!(i < 2 || i >= nx - 2 || j < 2 || j >= ny - 2)) continue;
        const long long g = cell_index(i, j, a.pitch);
        T v[6];
#pragma unroll
        for (int c = 0; c < 6; c++) v[c] = U[c * a.plane + g];
        write_ghosts(U, a.geo, a, i, j, v, tg);
    }
}

// mass bits (MB_*) of U for the 32 x TY tiles of tile rows [ty0, ty0 +
// gridDim.y): a CTA per tile, a warp per row
template <typename T, int TY>
__global__ void __launch_bounds__(32 * TY) mass_bits_kernel(const T *U, const T *R, int nx, int ny, int pitch,
                                                            long long plane, int ty0, unsigned short *mb)
{
    __shared__ unsigned int rows[TY];
    const int lane = threadIdx.x & 31, r = threadIdx.x >> 5;
    const int bx = blockIdx.x, ty = ty0 + blockIdx.y;
    const int i = bx * 32 + lane, j = ty * TY + r;
    bool m = false;
    if (i < nx && j < ny) {
        const long long g = cell_index(i, j, pitch);
        m = nonzero(U[g]) | nonzero(U[3 * plane + g]);
        if (R) m |= nonzero(R[g]) | nonzero(R[plane + g]);
    }
    const unsigned int b = __ballot_sync(0xffffffffu, m);
    if (lane == 0) rows[r] = b;
    __syncthreads();
    if (threadIdx.x == 0) mb[ty * gridDim.x + bx] = mass_bits<TY>(rows);
}

// release (h, phi_s, velocities) -> conserved U = J h (phi, phi v)
template <typename T>
__global__ void release_kernel(const double *src, int has_phi, int has_v, T *U, T *R, const T *geo, int nx, int ny,
                               int pitch, long long plane)
{
    const long long n = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / nx), i = (int)(e - (long long)j * nx);
        const long long g = cell_index(i, j, pitch);
        const double J = (double)geo[GC_J * plane + g];
        const double h = src[e];
        const double ph = has_phi ? src[n + e] : 0.5;
        const double U1 = J * h * ph, U4 = J * h * (1.0 - ph);
        const double vxs = (has_v & 1) ? src[2 * n + e] : 0.0, vys = (has_v & 2) ? src[3 * n + e] : 0.0;
        const double vxf = (has_v & 4) ? src[4 * n + e] : 0.0, vyf = (has_v & 8) ? src[5 * n + e] : 0.0;
        U[g] = (T)U1;
        U[plane + g] = (T)(U1 * vxs);
        U[2 * plane + g] = (T)(U1 * vys);
        U[3 * plane + g] = (T)U4;
        if (R) {
            R[g] = (T)(U1 - (double)(T)U1);
            R[plane + g] = (T)(U4 - (double)(T)U4);
        }
        U[4 * plane + g] = (T)(U4 * vxf);
        U[5 * plane + g] = (T)(U4 * vyf);
    }
}

// conserved -> output fields (h, phi_s, v_X^s, v_Y^s, v_X^f, v_Y^f)
template <typename T>
__global__ void prims_kernel(const T *U, const T *R, const T *geo, int nx, int ny, int pitch, long long plane,
                             double h_dry, double *dst)
{
    const long long n = (long long)nx * ny;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / nx), i = (int)(e - (long long)j * nx);
        const long long g = cell_index(i, j, pitch);
        const double J = (double)geo[GC_J * plane + g];
        double u[6];
        for (int c = 0; c < 6; c++) u[c] = (double)U[c * plane + g];
        if (R) {
            u[0] += (double)R[g];
            u[3] += (double)R[plane + g];
        }
        const double Ut = u[0] + u[3];
        const double h = Ut / J;
        const bool wet = h > h_dry;
        dst[e] = h;
        dst[n + e] = wet ? u[0] / Ut : 0.0;
        const bool ws = u[0] > J * h_dry, wf = u[3] > J * h_dry;
        dst[2 * n + e] = ws ? u[1] / u[0] : 0.0;
        dst[3 * n + e] = ws ? u[2] / u[0] : 0.0;
        dst[4 * n + e] = wf ? u[4] / u[3] : 0.0;
        dst[5 * n + e] = wf ? u[5] / u[3] : 0.0;
    }
}

template <typename T>
__global__ void budget_kernel(const T *U, const T *R, int nx, int j0, int j1, int pitch, long long plane, double *out)
{
    const long long n = (long long)nx * (j1 - j0);  // the rows [j0, j1)
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int j = j0 + (int)(e / nx), i = (int)(e - (long long)(j - j0) * nx);
        const long long g = cell_index(i, j, pitch);
#pragma unroll
        for (int c = 0; c < 6; c++) s[c] += (double)U[c * plane + g];
        if (R) {
            s[0] += (double)R[g];
            s[3] += (double)R[plane + g];
        }
    }
    __shared__ double w[6][32];
#pragma unroll
    for (int c = 0; c < 6; c++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
        if ((threadIdx.x & 31) == 0) w[c][threadIdx.x >> 5] = s[c];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += w[threadIdx.x][q];
        atomicAdd(&out[threadIdx.x], t);
    }
}

__global__ void validate_kernel(const double *src, long long n6, long long n, int *bad)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n6; e += (long long)gridDim.x * blockDim.x) {
        const double v = src[e];
        const int c = (int)(e / n);
        if (!isfinite(v) || ((c == 0 || c == 3) && v < 0.0)) atomicOr(bad, 1);
    }
}

// ---------------------------------------------------------------------------
// host helpers

static int ensure_stage_buf(moses_sim *s)
{
    if (!s->stage_buf) CK(cudaMalloc(&s->stage_buf, sizeof(double) * 6 * (size_t)s->nx * s->ny));
    return MOSES_OK;
}

static int read_ctl(moses_sim *s, Ctl *h)
{
    CK(cudaMemcpyAsync(h, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return MOSES_OK;
}

// after the state changed from the host: ghosts at the current time and a_max
template <typename T>
static int refresh_t(moses_sim *s)
{
    Ctl h;
    int rc = read_ctl(s, &h);
    if (rc) return rc;
    StageArgs<T> a = base_args<T>(s);
    const long long n = (long long)s->nx * s->ny;
    fill_ghosts_kernel<T><<<grid_for(n), 256, 0, s->stream>>>(a, (T *)s->U, h.t);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(&s->ctl->amax, 0, sizeof(unsigned long long), s->stream));
    // a new state clears a non-finite status left by an earlier step
    CK(cudaMemsetAsync(&s->ctl->status, 0, sizeof(s->ctl->status), s->stream));
    max_speed_kernel<T><<<grid_for(n), 256, 0, s->stream>>>((const T *)s->U, (const T *)s->geo, s->nx, s->own_j0,
                                                             s->own_j1, s->pitch, s->plane, &s->ctl->amax);
    CK(cudaGetLastError());
    return MOSES_OK;
}

static int refresh(moses_sim *s)
{
    return s->prec == MOSES_FP64 ? refresh_t<double>(s) : refresh_t<float>(s);
}

static int check_params(const moses_params *p, std::string &why)
{
    auto fin = [](double v) { return std::isfinite(v); };
    if (!(fin(p->g) && p->g > 0)) return why = "g must be > 0", 1;
    if (!(fin(p->eps) && p->eps > 0)) return why = "eps must be > 0", 1;
    if (!fin(p->eps_chi)) return why = "eps_chi must be finite", 1;
    if (!(fin(p->rho_s) && p->rho_s > 0)) return why = "rho_s must be > 0", 1;
    if (!(fin(p->rho_f) && p->rho_f >= 0 && p->rho_f < p->rho_s)) return why = "need 0 <= rho_f < rho_s", 1;
    if (!(fin(p->delta_b_deg) && p->delta_b_deg >= 0 && p->delta_b_deg < 90)) return why = "delta_b in [0, 90)", 1;
    if (p->k_mode != 0 && p->k_mode != 1) return why = "k_mode must be 0 or 1", 1;
    if (p->k_mode == 1) {
        if (!(fin(p->phi_int_deg) && p->phi_int_deg >= p->delta_b_deg && p->phi_int_deg < 90))
            return why = "k_mode 1 needs delta_b <= phi_int < 90 deg", 1;
        if (p->nu_f != 0.0 || p->scheme != MOSES_SCHEME_CENTRAL || p->recon != MOSES_RECON_MINMOD)
            return why = "k_mode 1 runs with the central flux, minmod and nu_f = 0", 1;
    }
    if (!(fin(p->c_d) && p->c_d >= 0)) return why = "c_d must be >= 0", 1;
    if (!(fin(p->nu_f) && p->nu_f >= 0)) return why = "nu_f must be >= 0", 1;
    if (!(fin(p->k_f) && p->k_f >= 0)) return why = "k_f must be >= 0", 1;
    if (!(fin(p->cfl) && p->cfl > 0)) return why = "cfl must be > 0", 1;
    if (!(fin(p->dt_max) && p->dt_max > 0)) return why = "dt_max must be > 0", 1;
    if (!(fin(p->h_dry) && p->h_dry >= 1e-30)) return why = "h_dry must be >= 1e-30", 1;
    for (int k = 0; k < 4; k++)
        if (p->bc[k] != MOSES_BC_CLOSED && p->bc[k] != MOSES_BC_TRANSMISSIVE) return why = "bc must be 0 or 1", 1;
    if (p->fluid_pg_mode != 0 && p->fluid_pg_mode != 1) return why = "fluid_pg_mode must be 0 or 1", 1;
    if (p->precision != MOSES_FP64 && p->precision != MOSES_FP32) return why = "precision must be 0 or 1", 1;
    if (p->scheme != MOSES_SCHEME_CENTRAL && p->scheme != MOSES_SCHEME_CENTRAL_UPWIND)
        return why = "scheme must be 0 or 1", 1;
    if (p->recon != MOSES_RECON_MINMOD && p->recon != MOSES_RECON_WENO3) return why = "recon must be 0 or 1", 1;
    if (p->rk != 0 && p->rk != 2 && p->rk != 3) return why = "rk must be 0, 2 or 3", 1;
    return 0;
}

static Phys make_phys(const moses_params *p, double dx, double dy)
{
    Phys f{};
    const double al = p->rho_f / p->rho_s;
    f.kap_s = p->eps * p->g * (1.0 - al) / 2.0;
    f.kap_f = p->eps * p->g / 2.0;
    f.half_g = p->g / 2.0;
    f.g_1ma = p->g * (1.0 - al);
    f.g = p->g;
    f.eps_chi = p->eps_chi;
    f.eps_alpha = p->eps * al;
    f.eps = p->eps;
    f.alpha = al;
    f.c_d = p->c_d;
    f.k_f = p->k_f;
    f.nu_f = p->nu_f;
    f.tan_delta = tan(p->delta_b_deg * M_PI / 180.0);
    f.h_dry = p->h_dry;
    f.cfl = p->cfl;
    f.dt_max = p->dt_max;
    f.dmin = dx < dy ? dx : dy;
    f.dx = dx;
    f.dy = dy;
    f.inv_dx = 1.0 / dx;
    f.inv_dy = 1.0 / dy;
    f.cell_area = dx * dy;
    f.pg_mode = p->fluid_pg_mode;
    f.scheme = p->scheme;
    f.recon = p->recon;
    f.rk = p->rk == 3 ? 3 : 2;
    for (int k = 0; k < 4; k++) f.bc[k] = p->bc[k];
    // Savage-Hutter earth-pressure coefficients (reading R10), from the
    // Mohr-Coulomb limit states of the solid against a bed of friction
    // delta_b: K = 2 sec^2(phi) (1 -/+ sqrt(1 - cos^2(phi) / cos^2(delta))) - 1
    f.k_mode = p->k_mode;
    f.K_act = f.K_pass = 1.0;
    if (p->k_mode == 1) {
        const double cphi = cos(p->phi_int_deg * M_PI / 180.0), cdel = cos(p->delta_b_deg * M_PI / 180.0);
        const double q = cphi * cphi / (cdel * cdel);
        const double root = sqrt(q < 1.0 ? 1.0 - q : 0.0);
        f.K_act = 2.0 / (cphi * cphi) * (1.0 - root) - 1.0;
        f.K_pass = 2.0 / (cphi * cphi) * (1.0 + root) - 1.0;
    }
    return f;
}

static void free_sim(moses_sim *s)
{
    if (!s) return;
    cudaFree(s->U);
    cudaFree(s->Us);
    cudaFree(s->Us2);
    cudaFree(s->wl);
    cudaFree(s->wl_n);
    cudaFree(s->tw[0]);
    cudaFree(s->tw[1]);
    cudaFree(s->zk);
    cudaFree(s->mb);
    cudaFree(s->geo);
    cudaFree(s->ctl);
    cudaFree(s->inflow_d);
    cudaFree(s->stage_buf);
    cudaFree(s->red);
    delete s;
}

// ---------------------------------------------------------------------------
// C-ABI (C linkage comes from the declarations in moses.h)

const char *moses_version(void) { return "moses-gb300 1.0 (sm_103a; FP64 and FP32 state forms)"; }

namespace {
// quiet NaN into columns [nx + 4, pitch) of `planes` planes of (ny + 4) rows
template <typename T>
__global__ void poison_kernel(T *buf, int planes, int nx, int ny, int pitch, long long plane)
{
    const int w = pitch - (nx + 2 * GH);
    const long long n = (long long)planes * (ny + 2 * GH) * w;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / w;  // plane * rows + row
        const int col = nx + 2 * GH + (int)(e - r * w);
        const int pl = (int)(r / (ny + 2 * GH)), row = (int)(r - (long long)pl * (ny + 2 * GH));
        buf[pl * plane + (long long)row * pitch + col] = (T)NAN;
    }
}
}  // namespace

int moses_debug_timeout(moses_sim *s, int on)
{
    const ZkReset zr{s};
    if (!s) return MOSES_EINVAL;
    s->dbg_stall = on ? 1 : 0;
    return MOSES_OK;
}

int moses_debug_poison(moses_sim *s)
{
    const ZkReset zr{s};
    if (!s) return MOSES_EINVAL;
    if (s->pitch == s->nx + 2 * GH) return MOSES_OK;  // no padding to poison
    const int sp = s->prec == MOSES_FP32 ? 8 : 6;
    const long long cells = (long long)(s->ny + 2 * GH) * (s->pitch - s->nx - 2 * GH);
    for (int q = 0; q < 3; q++) {
        void *buf = q == 0 ? s->U : q == 1 ? s->Us : s->geo;
        const int planes = q < 2 ? sp : geo_planes(s);
        if (s->prec == MOSES_FP64)
            poison_kernel<double><<<grid_for(planes * cells), 256, 0, s->stream>>>((double *)buf, planes, s->nx, s->ny,
                                                                                 s->pitch, s->plane);
        else
            poison_kernel<float><<<grid_for(planes * cells), 256, 0, s->stream>>>((float *)buf, planes, s->nx, s->ny,
                                                                                s->pitch, s->plane);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    return MOSES_OK;
}

namespace {
// the stage kernels' reciprocal and square roots beside CUDA's own results,
// one input per thread (moses_debug_math)
__global__ void math_kernel(const double *x, int n, double *out)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const double v = x[e];
        const float f = (float)v;
        out[0 * (long long)n + e] = moses::frcp(v);
        out[1 * (long long)n + e] = 1.0 / v;
        out[2 * (long long)n + e] = moses::fsqrt(v);
        out[3 * (long long)n + e] = sqrt(v);
        out[4 * (long long)n + e] = moses::frsqrt(v);
        out[5 * (long long)n + e] = rsqrt(v);
        out[6 * (long long)n + e] = (double)moses::frcp(f);
        out[7 * (long long)n + e] = (double)moses::fsqrt(f);
        out[8 * (long long)n + e] = (double)moses::frsqrt(f);
    }
}

// FP64 FMA throughput: eight independent FMA chains per thread, in registers
// only; b and c arrive at run time so nothing folds.  The sum of the chains
// is written where no input makes it land (a value no chain reaches), which
// keeps them live.
__global__ void fp64_fma_probe_kernel(double *sink, int iters, double b, double c)
{
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = 1e-3 * threadIdx.x + k;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = fma(a[k], b, c);
    }
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) t += a[k];
    if (t == -1.0) sink[0] = t;
}
}  // namespace

int moses_debug_fp64_rate(int reps, double *tflops)
{
    moses_sim *s = nullptr;  // errors go to moses_last_error(NULL)
    if (!tflops || reps < 1 || reps > 1000) return fail(s, MOSES_EINVAL, "need tflops and 1 <= reps <= 1000");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    double *sink = nullptr;
    CK(cudaMalloc(&sink, sizeof(double)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = sms * 4, threads = 256, iters = 4096;
    double best = 0.0;
    for (int r = 0; r <= reps && e == cudaSuccess; r++) {  // r = 0: warm-up
        cudaEventRecord(e0);
        fp64_fma_probe_kernel<<<blocks, threads>>>(sink, iters, 1.0000000001, 1e-12);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        const double fl = 2.0 * 8.0 * iters * (double)blocks * threads;
        if (e == cudaSuccess && r > 0 && ms > 0.0f) best = std::max(best, fl / (ms * 1e-3) / 1e12);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return fail(s, MOSES_ECUDA, std::string("moses_debug_fp64_rate: ") + cudaGetErrorString(e));
    *tflops = best;
    return MOSES_OK;
}

int moses_debug_math(const double *x, int n, double *out)
{
    moses_sim *s = nullptr;  // errors go to moses_last_error(NULL)
    if (!x || !out || n < 1 || n > (1 << 24)) return fail(s, MOSES_EINVAL, "need x, out and 1 <= n <= 2^24");
    double *d = nullptr;
    CK(cudaMalloc(&d, sizeof(double) * 10 * (size_t)n));
    cudaError_t e = cudaMemcpy(d, x, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        math_kernel<<<grid_for(n), 256>>>(d, n, d + n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d + n, sizeof(double) * 9 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(s, MOSES_ECUDA, std::string("moses_debug_math: ") + cudaGetErrorString(e));
    return MOSES_OK;
}

const char *moses_last_error(const moses_sim *s) { return s ? s->err.c_str() : g_create_err.c_str(); }

int moses_create(const double *dem, int nx, int ny, double dx, double dy, const moses_params *p, void *stream,
                 moses_sim **out)
{
    moses_sim *s = nullptr;
    if (!out) return fail(nullptr, MOSES_EINVAL, "out is NULL");
    *out = nullptr;
    if (!dem || !p) return fail(nullptr, MOSES_EINVAL, "dem and params must be non-NULL");
    if (nx < 1 || ny < 1) return fail(nullptr, MOSES_EINVAL, "nx and ny must be >= 1");
    if ((long long)nx * ny > (1ll << 31)) return fail(nullptr, MOSES_EINVAL, "grid larger than 2^31 cells");
    if (!(std::isfinite(dx) && std::isfinite(dy) && dx > 0 && dy > 0))
        return fail(nullptr, MOSES_EINVAL, "dx and dy must be finite and > 0");
    std::string why;
    if (check_params(p, why)) return fail(nullptr, MOSES_EINVAL, why);
    for (long long e = 0; e < (long long)nx * ny; e++)
        if (!std::isfinite(dem[e])) return fail(nullptr, MOSES_EINVAL, "DEM has non-finite values");

    s = new (std::nothrow) moses_sim();
    if (!s) return fail(nullptr, MOSES_ENOMEM, "host allocation failed");
    s->nx = nx;
    s->ny = ny;
    s->own_j0 = 0;
    s->own_j1 = ny;
    s->dx = dx;
    s->dy = dy;
    s->p = *p;
    s->ph = make_phys(p, dx, dy);
    s->prec = p->precision;
    s->esz = s->prec == MOSES_FP64 ? 8 : 4;
    s->stream = (cudaStream_t)stream;
    s->pitch = ((nx + 2 * GH) + 31) / 32 * 32;
    s->plane = (long long)s->pitch * (ny + 2 * GH);
    auto bail = [&](int rc) {
        g_create_err = s->err;
        free_sim(s);
        return rc;
    };
    const size_t st = (s->prec == MOSES_FP32 ? 8 : 6) * (size_t)s->plane * s->esz;
    cudaError_t e;
    if ((e = cudaMalloc(&s->U, st)) != cudaSuccess || (e = cudaMalloc(&s->Us, st)) != cudaSuccess ||
        (e = cudaMalloc(&s->geo, (size_t)geo_planes(s) * s->plane * s->esz)) != cudaSuccess ||
        (s->ph.rk == 3 && (e = cudaMalloc(&s->Us2, st)) != cudaSuccess) ||
        (e = cudaMalloc(&s->wl, sizeof(int) * (size_t)((nx + 31) / 32) * ((ny + 3) / 4))) != cudaSuccess ||
        (e = cudaMalloc(&s->wl_n, 2 * sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaMalloc(&s->tw[0], (size_t)((nx + 31) / 32) * ((ny + 3) / 4))) != cudaSuccess ||
        (e = cudaMalloc(&s->tw[1], (size_t)((nx + 31) / 32) * ((ny + 3) / 4))) != cudaSuccess ||
        (e = cudaMalloc(&s->zk, 3 * (size_t)((nx + 31) / 32) * ((ny + 3) / 4))) != cudaSuccess ||
        (e = cudaMalloc(&s->mb, 3 * sizeof(unsigned short) * (size_t)((nx + 31) / 32) * ((ny + 3) / 4))) !=
            cudaSuccess ||
        (e = cudaMalloc(&s->ctl, sizeof(Ctl))) != cudaSuccess ||
        (e = cudaMalloc(&s->inflow_d, sizeof(InflowSeg) * MAX_INFLOW)) != cudaSuccess ||
        (e = cudaMalloc(&s->red, 8 * sizeof(double))) != cudaSuccess) {
        s->err = std::string("device allocation failed: ") + cudaGetErrorString(e);
        return bail(e == cudaErrorMemoryAllocation ? MOSES_ENOMEM : MOSES_ECUDA);
    }
    if ((e = cudaMemsetAsync(s->U, 0, st, s->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(s->Us, 0, st, s->stream)) != cudaSuccess ||
        (s->Us2 && (e = cudaMemsetAsync(s->Us2, 0, st, s->stream)) != cudaSuccess) ||
        (e = cudaMemsetAsync(s->wl_n, 0, 2 * sizeof(unsigned int), s->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(s->geo, 0, (size_t)geo_planes(s) * s->plane * s->esz, s->stream)) != cudaSuccess) {
        s->err = std::string("memset: ") + cudaGetErrorString(e);
        return bail(MOSES_ECUDA);
    }
    Ctl c{};
    if ((e = cudaMemcpyAsync(s->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s->stream)) != cudaSuccess) {
        s->err = std::string("ctl: ") + cudaGetErrorString(e);
        return bail(MOSES_ECUDA);
    }
    // geometry pass
    double *d_dem = nullptr, *d_ext = nullptr;
    const size_t nd = (size_t)nx * ny, ne = (size_t)(nx + 6) * (ny + 6);
    if ((e = cudaMalloc(&d_dem, nd * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&d_ext, ne * sizeof(double))) != cudaSuccess) {
        cudaFree(d_dem);
        s->err = std::string("device allocation failed: ") + cudaGetErrorString(e);
        return bail(MOSES_ENOMEM);
    }
    e = cudaMemcpyAsync(d_dem, dem, nd * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) {
        extend_dem_kernel<<<grid_for((long long)ne), 256, 0, s->stream>>>(d_dem, nx, ny, d_ext);
        const long long ng = (long long)(nx + 4) * (ny + 4);
        if (s->prec == MOSES_FP64)
            geometry_kernel<double><<<grid_for(ng), 256, 0, s->stream>>>(d_ext, nx, ny, s->pitch, s->plane, dx, dy,
                                                                         s->ph, (double *)s->geo, has_slopes(s));
        else
            geometry_kernel<float><<<grid_for(ng), 256, 0, s->stream>>>(d_ext, nx, ny, s->pitch, s->plane, dx, dy,
                                                                        s->ph, (float *)s->geo, 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(d_dem);
    cudaFree(d_ext);
    if (e != cudaSuccess) {
        s->err = std::string("geometry pass: ") + cudaGetErrorString(e);
        return bail(MOSES_ECUDA);
    }
    s->have_state = true;  // dry state at t = 0
    int rc = refresh(s);
    if (rc) return bail(rc);
    *out = s;
    return MOSES_OK;
}

void moses_destroy(moses_sim *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    free_sim(s);
}

static int upload_dense(moses_sim *s, const double *host6)
{
    int rc = ensure_stage_buf(s);
    if (rc) return rc;
    CK(cudaMemcpyAsync(s->stage_buf, host6, sizeof(double) * 6 * (size_t)s->nx * s->ny, cudaMemcpyHostToDevice,
                       s->stream));
    return MOSES_OK;
}

int moses_set_release(moses_sim *s, const double *h, const double *phi_s, const double *vx_s, const double *vy_s,
                      const double *vx_f, const double *vy_f)
{
    const ZkReset zr{s};
    if (!s) return MOSES_EINVAL;
    if (!h) return fail(s, MOSES_EINVAL, "h must be non-NULL");
    const long long n = (long long)s->nx * s->ny;
    for (long long e = 0; e < n; e++) {
        if (!(std::isfinite(h[e]) && h[e] >= 0)) return fail(s, MOSES_EINVAL, "h must be finite and >= 0");
        if (phi_s && !(phi_s[e] >= 0 && phi_s[e] <= 1)) return fail(s, MOSES_EINVAL, "phi_s must be in [0, 1]");
    }
    const double *v[4] = {vx_s, vy_s, vx_f, vy_f};
    for (int q = 0; q < 4; q++)
        if (v[q])
            for (long long e = 0; e < n; e++)
                if (!std::isfinite(v[q][e])) return fail(s, MOSES_EINVAL, "velocities must be finite");
    int rc = ensure_stage_buf(s);
    if (rc) return rc;
    const size_t b = sizeof(double) * (size_t)n;
    CK(cudaMemcpyAsync(s->stage_buf, h, b, cudaMemcpyHostToDevice, s->stream));
    if (phi_s) CK(cudaMemcpyAsync(s->stage_buf + n, phi_s, b, cudaMemcpyHostToDevice, s->stream));
    int has_v = 0;
    for (int q = 0; q < 4; q++)
        if (v[q]) {
            CK(cudaMemcpyAsync(s->stage_buf + (2 + q) * n, v[q], b, cudaMemcpyHostToDevice, s->stream));
            has_v |= 1 << q;
        }
    if (s->prec == MOSES_FP64)
        release_kernel<double><<<grid_for(n), 256, 0, s->stream>>>(s->stage_buf, phi_s != nullptr, has_v,
                                                                   (double *)s->U, nullptr, (const double *)s->geo, s->nx,
                                                                   s->ny, s->pitch, s->plane);
    else
        release_kernel<float><<<grid_for(n), 256, 0, s->stream>>>(s->stage_buf, phi_s != nullptr, has_v,
                                                                  (float *)s->U, rem<float>(s, s->U), (const float *)s->geo, s->nx,
                                                                  s->ny, s->pitch, s->plane);
    CK(cudaGetLastError());
    s->have_state = true;
    rc = refresh(s);
    if (rc) return rc;
    CK(cudaStreamSynchronize(s->stream));
    return MOSES_OK;
}

int moses_set_inflow(moses_sim *s, int side, int i0, int i1, int npts, const double *t, const double *Q,
                     const double *phi_s)
{
    const ZkReset zr{s};
    if (!s) return MOSES_EINVAL;
    if (s->n_inflow >= MAX_INFLOW) return fail(s, MOSES_EINVAL, "at most 8 inflow segments");
    if (side < 0 || side > 3) return fail(s, MOSES_EINVAL, "side must be 0..3");
    const int len = side < 2 ? s->ny : s->nx;
    if (i0 < 0 || i1 > len || i1 <= i0) return fail(s, MOSES_EINVAL, "segment [i0, i1) outside the side");
    if (npts < 1 || npts > MAX_HYD || !t || !Q || !phi_s) return fail(s, MOSES_EINVAL, "need 1..64 hydrograph points");
    for (int k = 0; k < npts; k++) {
        if (!(std::isfinite(t[k]) && std::isfinite(Q[k]) && Q[k] >= 0 && phi_s[k] >= 0 && phi_s[k] <= 1))
            return fail(s, MOSES_EINVAL, "hydrograph values must be finite, Q >= 0, phi_s in [0, 1]");
        if (k && t[k] < t[k - 1]) return fail(s, MOSES_EINVAL, "hydrograph times must not decrease");
    }
    for (int f = 0; f < s->n_inflow; f++)
        if (s->inflow_h[f].side == side && i0 < s->inflow_h[f].i1 && s->inflow_h[f].i0 < i1)
            return fail(s, MOSES_EINVAL, "inflow segments overlap");
    InflowSeg &g = s->inflow_h[s->n_inflow];
    memset(&g, 0, sizeof(g));
    g.side = side;
    g.i0 = i0;
    g.i1 = i1;
    g.npts = npts;
    for (int k = 0; k < npts; k++) {
        g.t[k] = t[k];
        g.Q[k] = Q[k];
        g.phi[k] = phi_s[k];
    }
    CK(cudaMemcpyAsync(s->inflow_d + s->n_inflow, &g, sizeof(InflowSeg), cudaMemcpyHostToDevice, s->stream));
    s->n_inflow++;
    int rc = refresh(s);
    if (rc) return rc;
    CK(cudaStreamSynchronize(s->stream));
    return MOSES_OK;
}

template <typename T>
static int launch_steps(moses_sim *s, int nsteps, double *stage_ms = nullptr)
{
    // the stages of one step: the two-step modified Euler (U -> Us -> U), or
    // the three-stage SSP Runge-Kutta (U -> Us -> Us2 -> U)
    StageArgs<T> a[3] = {base_args<T>(s), base_args<T>(s), base_args<T>(s)};
    const bool rk3 = s->ph.rk == 3;
    const int ns = rk3 ? 3 : 2;
    void *out[3] = {s->Us, rk3 ? s->Us2 : s->U, s->U};
    void *in[3] = {s->U, s->Us, s->Us2};
    // the known-zero tile flags of the output buffers: the plain form's
    // classification keeps them (the model options test each tile in the
    // stage kernel, which writes every tile)
    const size_t nt = (size_t)((s->nx + 31) / 32) * ((s->ny + 3) / 4);
    const bool zk_on = !(s->ph.nu_f > 0.0) && s->ph.scheme != 1 && s->ph.recon != 1;
    if (zk_on && !s->zk_valid) CK(cudaMemsetAsync(s->zk, 0, 3 * nt, s->stream));
    // U's mass bits describe U where the flags do (the last stepping launches
    // wrote both); the copy-wait test needs the data classification
    const bool mb_first = s->zk_valid && zk_on && !s->dbg_stall;
    s->zk_valid = false;  // until the launches below are in
    auto bufno = [&](const void *b) { return b == s->U ? 0 : b == s->Us ? 1 : 2; };
    for (int q = 0; q < ns; q++) {
        a[q].Uin = (const T *)in[q];
        a[q].Uout = (T *)out[q];
        a[q].Rin = rem<T>(s, in[q]);
        a[q].Rout = rem<T>(s, out[q]);
        a[q].stage = q == 0 ? 1 : 2;
        if (q > 0) {
            a[q].Un = (const T *)s->U;
            a[q].Rn = rem<T>(s, s->U);
        }
        a[q].want_amax = q == ns - 1;
        a[q].wl = s->wl;
        a[q].wl_n = s->wl_n;
        // the first stage classifies from the data or the mass bits, the later
        // ones from the mass bits (the stage-before flags only where the bits are off)
        a[q].tw_next = s->tw[q % 2];
        a[q].tw_prev = q > 0 && !zk_on ? s->tw[(q - 1) % 2] : nullptr;
        if (zk_on) {
            a[q].zk = s->zk + nt * bufno(out[q]);
            a[q].mb_in = s->mb + nt * bufno(in[q]);
            a[q].mb_out = s->mb + nt * bufno(out[q]);
            if (q > 0) a[q].mb_n = s->mb;
            a[q].mb_ok = q > 0 || mb_first;
        }
        if (rk3) {
            a[q].rk3 = q + 1;
            a[q].rk3_bw = q == 2 ? 2.0 / 3.0 : 1.0 / 6.0;
        }
    }
    // the later steps of this call: the first stage from the bits the step before wrote
    StageArgs<T> a0_next = a[0];
    if (zk_on && !s->dbg_stall) a0_next.mb_ok = 1;
    if (stage_ms) {
        // events around every launch; the first stage in stage_ms[0], the others in stage_ms[1]
        cudaEvent_t ev[4];
        for (int q = 0; q < 4; q++) CK(cudaEventCreate(&ev[q]));
        double acc[2] = {0.0, 0.0};
        int rc = 0;
        for (int k = 0; k < nsteps && rc == 0; k++) {
            CK(cudaEventRecord(ev[0], s->stream));
            for (int q = 0; q < ns && rc == 0; q++) {
                rc = launch_stage<T>(q == 0 && k > 0 ? a0_next : a[q], s->tile, s->stream);
                CK(cudaEventRecord(ev[q + 1], s->stream));
            }
            CK(cudaEventSynchronize(ev[ns]));
            float m1 = 0.f, m2 = 0.f;
            CK(cudaEventElapsedTime(&m1, ev[0], ev[1]));
            CK(cudaEventElapsedTime(&m2, ev[1], ev[ns]));
            acc[0] += m1;
            acc[1] += m2;
        }
        for (int q = 0; q < 4; q++) cudaEventDestroy(ev[q]);
        if (rc) return fail(s, MOSES_ECUDA, std::string("stage launch: ") + cudaGetErrorString(cudaGetLastError()));
        stage_ms[0] = acc[0];
        stage_ms[1] = acc[1];
        s->zk_valid = zk_on;
        return MOSES_OK;
    }
    for (int k = 0; k < nsteps; k++) {
        int rc = 0;
        for (int q = 0; q < ns && rc == 0; q++) rc = launch_stage<T>(q == 0 && k > 0 ? a0_next : a[q], s->tile, s->stream);
        if (rc) return fail(s, MOSES_ECUDA, std::string("stage launch: ") + cudaGetErrorString(cudaGetLastError()));
    }
    s->zk_valid = zk_on;
    return MOSES_OK;
}

static int set_mode(moses_sim *s, double dt_fixed, double t_end)
{
    CK(cudaMemcpyAsync(&s->ctl->dt_fixed, &dt_fixed, sizeof(double), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(&s->ctl->t_end, &t_end, sizeof(double), cudaMemcpyHostToDevice, s->stream));
    return MOSES_OK;
}

static int run_steps(moses_sim *s, int nsteps, double dt_fixed, double t_end, double *t_out,
                     double *stage_ms = nullptr)
{
    if (!s) return MOSES_EINVAL;
    if (nsteps < 0) return fail(s, MOSES_EINVAL, "nsteps must be >= 0");
    if (!s->have_state) return fail(s, MOSES_ESTATE, "no state");
    int rc = set_mode(s, dt_fixed, t_end);
    if (rc) return rc;
    rc = s->prec == MOSES_FP64 ? launch_steps<double>(s, nsteps, stage_ms) : launch_steps<float>(s, nsteps, stage_ms);
    if (rc) return rc;
    Ctl h;
    rc = read_ctl(s, &h);
    if (rc) return rc;
    if (t_out) *t_out = h.t;
    if (h.status & (STATUS_TIMEOUT | STATUS_NONFINITE)) zk_reset(s);  // a classification may have stopped early
    if (h.status & STATUS_TIMEOUT) return fail(s, MOSES_ETIMEOUT, "a bounded device-side wait gave up");
    if (h.status & STATUS_NONFINITE) return fail(s, MOSES_ENONFINITE, "state or time step became non-finite");
    return MOSES_OK;
}

int moses_step(moses_sim *s, int nsteps, double *t_out) { return run_steps(s, nsteps, 0.0, 0.0, t_out); }

int moses_step_timed(moses_sim *s, int nsteps, double *t_out, double *stage_ms)
{
    if (!s || !stage_ms) return MOSES_EINVAL;
    return run_steps(s, nsteps, 0.0, 0.0, t_out, stage_ms);
}

int moses_set_tile(moses_sim *s, int tile)
{
    const ZkReset zr{s};
    if (!s) return MOSES_EINVAL;
    if (tile < 0 || tile >= MOSES_NTILES) return fail(s, MOSES_EINVAL, "tile must be one of MOSES_TILE_*");
    s->tile = tile;
    return MOSES_OK;
}

namespace {
std::mutex g_tune_mu;
std::map<std::array<int, 5>, int> g_tune_cache;  // (device, SMs, precision, nx, ny) -> tile

// the first stage of a step as moses_step launches it in its steady state
// (wet-tile list, known-zero flags of U*, mass bits of U), from the current
// state into the scratch buffer; `steady` false: the first such stage after a
// state change, which classifies from the data and writes U's mass bits.  It
// also touches the control block (time step, budgets), which the caller
// restores
template <typename T>
int probe_stage(moses_sim *s, int tile, bool steady)
{
    const size_t nt = (size_t)((s->nx + 31) / 32) * ((s->ny + 3) / 4);
    StageArgs<T> a = base_args<T>(s);
    a.Uin = (const T *)s->U;
    a.Uout = (T *)s->Us;
    a.Rin = rem<T>(s, s->U);
    a.Rout = rem<T>(s, s->Us);
    a.stage = 1;
    a.wl = s->wl;
    a.wl_n = s->wl_n;
    a.tw_next = s->tw[0];
    a.zk = s->zk + nt;
    a.mb_in = s->mb;
    a.mb_out = s->mb + nt;
    a.mb_ok = steady;
    return launch_stage<T>(a, tile, s->stream);
}
}  // namespace

int moses_autotune(moses_sim *s, int reps, int *tile_out, double *ms_out)
{
    const ZkReset zr{s};
    if (!s) return MOSES_EINVAL;
    if (reps < 0) return fail(s, MOSES_EINVAL, "reps must be >= 0");
    if (reps == 0) reps = 5;
    if (!s->have_state) return fail(s, MOSES_ESTATE, "no state");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const std::array<int, 5> key{dev, sms, s->prec, s->nx, s->ny};
    if (!ms_out) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            s->tile = it->second;
            if (tile_out) *tile_out = s->tile;
            return MOSES_OK;
        }
    }
    Ctl h;
    int rc = read_ctl(s, &h);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double ms[MOSES_NTILES];
    int best = 0;
    const size_t nt = (size_t)((s->nx + 31) / 32) * ((s->ny + 3) / 4);
    const bool listed = !(s->ph.nu_f > 0.0) && s->ph.scheme != 1 && s->ph.recon != 1;
    // two rounds over the shapes, each launch timed alone: the fastest launch
    // of each shape counts (the shapes often lie within a few per cent, and
    // one slow launch should not decide)
    for (int t = 0; t < MOSES_NTILES; t++) ms[t] = 1e30;
    for (int round = 0; round < 2 && rc == 0; round++)
        for (int t = 0; t < MOSES_NTILES && rc == 0; t++) {
            // an untimed first stage sets up the shape's flags and mass bits; the
            // timed ones then run as the steps of a run do
            if (cudaMemsetAsync(s->zk, 0, 3 * nt, s->stream) != cudaSuccess) rc = -1;
            for (int r = 0; r <= reps && rc == 0; r++) {
                const bool steady = r > 0 && listed;
                if (r > 0) cudaEventRecord(e0, s->stream);
                rc = s->prec == MOSES_FP64 ? probe_stage<double>(s, t, steady) : probe_stage<float>(s, t, steady);
                if (r == 0 || rc) continue;
                cudaEventRecord(e1, s->stream);
                float f = 0.0f;
                if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&f, e0, e1) == cudaSuccess)
                    ms[t] = std::min(ms[t], (double)f);
                else
                    rc = -1;
            }
        }
    for (int t = 1; t < MOSES_NTILES; t++)
        if (ms[t] < ms[best]) best = t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return fail(s, MOSES_ECUDA, "autotune launch failed");
    // the probes advanced nothing: put the control block back as it was
    CK(cudaMemcpyAsync(s->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->tile = best;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    if (tile_out) *tile_out = best;
    if (ms_out)
        for (int t = 0; t < MOSES_NTILES; t++) ms_out[t] = ms[t];
    return MOSES_OK;
}

int moses_step_dt(moses_sim *s, int nsteps, double dt, double *t_out)
{
    if (!s) return MOSES_EINVAL;
    if (!(std::isfinite(dt) && dt > 0)) return fail(s, MOSES_EINVAL, "dt must be finite and > 0");
    return run_steps(s, nsteps, dt, 0.0, t_out);
}

int moses_run_until(moses_sim *s, double t_end, int max_steps, int *nsteps_out)
{
    if (!s) return MOSES_EINVAL;
    if (!std::isfinite(t_end)) return fail(s, MOSES_EINVAL, "t_end must be finite");
    Ctl h;
    int rc = read_ctl(s, &h);
    if (rc) return rc;
    const long long s0 = h.steps;
    const int chunk = 64;
    while (h.t < t_end && h.steps - s0 < max_steps) {
        const int n = (int)std::min<long long>(chunk, max_steps - (h.steps - s0));
        rc = run_steps(s, n, 0.0, t_end, nullptr);
        if (rc) return rc;
        rc = read_ctl(s, &h);
        if (rc) return rc;
        if (h.t >= t_end) break;
    }
    if (nsteps_out) *nsteps_out = (int)(h.steps - s0);
    // steps after reaching t_end would have dt = 0: count only real ones
    return MOSES_OK;
}

int moses_next_dt(moses_sim *s, double *dt, double *t)
{
    if (!s) return MOSES_EINVAL;
    Ctl h;
    int rc = read_ctl(s, &h);
    if (rc) return rc;
    const double am = *reinterpret_cast<double *>(&h.amax);
    double d = (am > 0.0) ? s->ph.cfl * s->ph.dmin / am : s->ph.dt_max;
    if (d > s->ph.dt_max) d = s->ph.dt_max;
    if (dt) *dt = d;
    if (t) *t = h.t;
    return MOSES_OK;
}

int moses_max_speed(moses_sim *s, double *amax)
{
    if (!s || !amax) return MOSES_EINVAL;
    Ctl h;
    int rc = read_ctl(s, &h);
    if (rc) return rc;
    *amax = *reinterpret_cast<double *>(&h.amax);
    return MOSES_OK;
}

int moses_get_conserved_device(moses_sim *s, double *U_device)
{
    if (!s || !U_device) return MOSES_EINVAL;
    const long long n = (long long)s->nx * s->ny;
    if (s->prec == MOSES_FP64)
        pack_kernel<double><<<grid_for(6 * n), 256, 0, s->stream>>>((const double *)s->U, nullptr, U_device, s->nx, s->ny,
                                                                    s->pitch, s->plane);
    else
        pack_kernel<float><<<grid_for(6 * n), 256, 0, s->stream>>>((const float *)s->U, rem<float>(s, s->U), U_device, s->nx, s->ny,
                                                                   s->pitch, s->plane);
    CK(cudaGetLastError());
    return MOSES_OK;
}

int moses_get_conserved(moses_sim *s, double *U)
{
    if (!s || !U) return MOSES_EINVAL;
    int rc = ensure_stage_buf(s);
    if (rc) return rc;
    rc = moses_get_conserved_device(s, s->stage_buf);
    if (rc) return rc;
    CK(cudaMemcpyAsync(U, s->stage_buf, sizeof(double) * 6 * (size_t)s->nx * s->ny, cudaMemcpyDeviceToHost,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return MOSES_OK;
}

static int set_from_device_buf(moses_sim *s, const double *src)
{
    const long long n = (long long)s->nx * s->ny;
    CK(cudaMemsetAsync(s->red, 0, sizeof(int), s->stream));
    validate_kernel<<<grid_for(6 * n), 256, 0, s->stream>>>(src, 6 * n, n, (int *)s->red);
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, s->red, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (bad) return fail(s, MOSES_EINVAL, "U must be finite with U1, U4 >= 0");
    if (s->prec == MOSES_FP64)
        unpack_kernel<double><<<grid_for(6 * n), 256, 0, s->stream>>>(src, (double *)s->U, nullptr, s->nx, s->ny, s->pitch,
                                                                      s->plane);
    else
        unpack_kernel<float><<<grid_for(6 * n), 256, 0, s->stream>>>(src, (float *)s->U, rem<float>(s, s->U), s->nx, s->ny, s->pitch,
                                                                     s->plane);
    CK(cudaGetLastError());
    s->have_state = true;
    return refresh(s);
}

int moses_set_conserved_device(moses_sim *s, const double *U_device)
{
    const ZkReset zr{s};
    if (!s || !U_device) return MOSES_EINVAL;
    return set_from_device_buf(s, U_device);
}

int moses_set_conserved(moses_sim *s, const double *U)
{
    const ZkReset zr{s};
    if (!s || !U) return MOSES_EINVAL;
    int rc = upload_dense(s, U);
    if (rc) return rc;
    rc = set_from_device_buf(s, s->stage_buf);
    if (rc) return rc;
    CK(cudaStreamSynchronize(s->stream));
    return MOSES_OK;
}

// ---------------------------------------------------------------------------
// One strip of a row-decomposed domain: owned rows, row exchange, the CFL
// maximum over all strips.

int moses_set_owned_rows(moses_sim *s, int j0, int j1)
{
    if (!s) return MOSES_EINVAL;
    if (j0 < 0 || j1 > s->ny || j1 <= j0) return fail(s, MOSES_EINVAL, "owned rows must satisfy 0 <= j0 < j1 <= ny");
    s->own_j0 = j0;
    s->own_j1 = j1;
    // the CFL maximum of the current state over the own rows (the rows near
    // a window's inner edges see an extrapolated bed)
    if (!s->have_state) return MOSES_OK;
    CK(cudaMemsetAsync(&s->ctl->amax, 0, sizeof(unsigned long long), s->stream));
    const long long n = (long long)s->nx * (j1 - j0);
    if (s->prec == MOSES_FP64)
        max_speed_kernel<double><<<grid_for(n), 256, 0, s->stream>>>((const double *)s->U, (const double *)s->geo,
                                                                     s->nx, j0, j1, s->pitch, s->plane, &s->ctl->amax);
    else
        max_speed_kernel<float><<<grid_for(n), 256, 0, s->stream>>>((const float *)s->U, (const float *)s->geo, s->nx,
                                                                    j0, j1, s->pitch, s->plane, &s->ctl->amax);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
    return MOSES_OK;
}

int moses_row_planes(const moses_sim *s) { return s ? (s->prec == MOSES_FP32 ? 8 : 6) : 0; }

int moses_get_rows_device(moses_sim *s, int j0, int nrows, double *rows_device)
{
    if (!s || !rows_device) return MOSES_EINVAL;
    if (j0 < 0 || nrows < 1 || j0 + nrows > s->ny) return fail(s, MOSES_EINVAL, "rows outside the grid");
    const long long n = (long long)moses_row_planes(s) * s->nx * nrows;
    if (s->prec == MOSES_FP64)
        rows_pack_kernel<double><<<grid_for(n), 256, 0, s->stream>>>((const double *)s->U, nullptr, rows_device, s->nx,
                                                                     j0, nrows, s->pitch, s->plane);
    else
        rows_pack_kernel<float><<<grid_for(n), 256, 0, s->stream>>>((const float *)s->U, rem<float>(s, s->U),
                                                                    rows_device, s->nx, j0, nrows, s->pitch, s->plane);
    CK(cudaGetLastError());
    return MOSES_OK;
}

namespace {
template <typename T, int TY>
int rows_mass_bits(moses_sim *s, int ty0, int ty1)
{
    const dim3 grid((s->nx + 31) / 32, ty1 - ty0);
    mass_bits_kernel<T, TY><<<grid, 32 * TY, 0, s->stream>>>((const T *)s->U, rem<T>(s, s->U), s->nx, s->ny, s->pitch,
                                                             s->plane, ty0, s->mb);
    CK(cudaGetLastError());
    return MOSES_OK;
}

// after rows [j0, j1) of U were replaced: their ghosts; the known-zero flags
// and mass bits of the tiles they touch (the stepping launches' own records
// of U stay valid for every other tile)
template <typename T>
int rows_replaced(moses_sim *s, int j0, int j1)
{
    StageArgs<T> a = base_args<T>(s);
    fill_ghosts_rows_kernel<T><<<grid_for((long long)s->nx * (j1 - j0)), 256, 0, s->stream>>>(a, (T *)s->U, j0, j1);
    CK(cudaGetLastError());
    const int TY = tile_rows(s->tile);
    const int gx = (s->nx + 31) / 32, ty0 = j0 / TY, ty1 = (j1 - 1) / TY + 1;
    CK(cudaMemsetAsync(s->zk + (size_t)ty0 * gx, 0, (size_t)(ty1 - ty0) * gx, s->stream));  // U's flags
    switch (TY) {
    case 4: return rows_mass_bits<T, 4>(s, ty0, ty1);
    case 16: return rows_mass_bits<T, 16>(s, ty0, ty1);
    default: return rows_mass_bits<T, 8>(s, ty0, ty1);
    }
}
}  // namespace

int moses_set_rows_device(moses_sim *s, int j0, int nrows, const double *rows_device)
{
    if (!s || !rows_device) return MOSES_EINVAL;
    if (!s->have_state) return fail(s, MOSES_ESTATE, "no state");
    if (j0 < 0 || nrows < 1 || j0 + nrows > s->ny) return fail(s, MOSES_EINVAL, "rows outside the grid");
    const long long n = (long long)moses_row_planes(s) * s->nx * nrows;
    if (s->prec == MOSES_FP64)
        rows_unpack_kernel<double><<<grid_for(n), 256, 0, s->stream>>>(rows_device, (double *)s->U, nullptr, s->nx, j0,
                                                                       nrows, s->pitch, s->plane);
    else
        rows_unpack_kernel<float><<<grid_for(n), 256, 0, s->stream>>>(rows_device, (float *)s->U, rem<float>(s, s->U),
                                                                      s->nx, j0, nrows, s->pitch, s->plane);
    CK(cudaGetLastError());
    return s->prec == MOSES_FP64 ? rows_replaced<double>(s, j0, j0 + nrows) : rows_replaced<float>(s, j0, j0 + nrows);
}

int moses_set_max_speed(moses_sim *s, double amax)
{
    if (!s) return MOSES_EINVAL;
    if (!(std::isfinite(amax) && amax >= 0.0)) return fail(s, MOSES_EINVAL, "amax must be finite and >= 0");
    const double v = amax + 0.0;  // -0 -> +0: the step reads the IEEE bits as a non-negative double
    CK(cudaMemcpyAsync(&s->ctl->amax, &v, sizeof(double), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return MOSES_OK;
}

int moses_get_state(moses_sim *s, double *h, double *phi_s, double *vx_s, double *vy_s, double *vx_f, double *vy_f)
{
    if (!s) return MOSES_EINVAL;
    int rc = ensure_stage_buf(s);
    if (rc) return rc;
    const long long n = (long long)s->nx * s->ny;
    if (s->prec == MOSES_FP64)
        prims_kernel<double><<<grid_for(n), 256, 0, s->stream>>>((const double *)s->U, nullptr, (const double *)s->geo, s->nx,
                                                                 s->ny, s->pitch, s->plane, s->ph.h_dry,
                                                                 s->stage_buf);
    else
        prims_kernel<float><<<grid_for(n), 256, 0, s->stream>>>((const float *)s->U, rem<float>(s, s->U), (const float *)s->geo, s->nx,
                                                                s->ny, s->pitch, s->plane, s->ph.h_dry, s->stage_buf);
    CK(cudaGetLastError());
    double *dst[6] = {h, phi_s, vx_s, vy_s, vx_f, vy_f};
    for (int q = 0; q < 6; q++)
        if (dst[q])
            CK(cudaMemcpyAsync(dst[q], s->stage_buf + q * n, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return MOSES_OK;
}

int moses_stage(moses_sim *s, double t, double dt, double *U_out)
{
    const ZkReset zr{s};
    if (!s || !U_out) return MOSES_EINVAL;
    if (!(std::isfinite(dt) && dt >= 0 && std::isfinite(t))) return fail(s, MOSES_EINVAL, "bad t or dt");
    int rc = ensure_stage_buf(s);
    if (rc) return rc;
    // ghosts of the current state at time t
    Ctl h;
    rc = read_ctl(s, &h);
    if (rc) return rc;
    const double t_saved = h.t;
    CK(cudaMemcpyAsync(&s->ctl->t, &t, sizeof(double), cudaMemcpyHostToDevice, s->stream));
    rc = refresh(s);
    if (rc) return rc;
    CK(cudaMemcpyAsync(&s->ctl->t, &t_saved, sizeof(double), cudaMemcpyHostToDevice, s->stream));
    if (s->prec == MOSES_FP64) {
        StageArgs<double> a = base_args<double>(s);
        a.Uin = (const double *)s->U;
        a.Uout = (double *)s->Us;
        a.stage = 1;
        a.debug_stage = 1;
        a.dbg_t = t;
        a.dbg_dt = dt;
        rc = launch_stage<double>(a, s->tile, s->stream);
        if (rc == 0)
            pack_kernel<double><<<grid_for(6LL * s->nx * s->ny), 256, 0, s->stream>>>(
                (const double *)s->Us, nullptr, s->stage_buf, s->nx, s->ny, s->pitch, s->plane);
    } else {
        StageArgs<float> a = base_args<float>(s);
        a.Uin = (const float *)s->U;
        a.Uout = (float *)s->Us;
        a.Rin = rem<float>(s, s->U);
        a.Rout = rem<float>(s, s->Us);
        a.stage = 1;
        a.debug_stage = 1;
        a.dbg_t = t;
        a.dbg_dt = dt;
        rc = launch_stage<float>(a, s->tile, s->stream);
        if (rc == 0)
            pack_kernel<float><<<grid_for(6LL * s->nx * s->ny), 256, 0, s->stream>>>(
                (const float *)s->Us, rem<float>(s, s->Us), s->stage_buf, s->nx, s->ny, s->pitch, s->plane);
    }
    if (rc) return fail(s, MOSES_ECUDA, "stage launch failed");
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(U_out, s->stage_buf, sizeof(double) * 6 * (size_t)s->nx * s->ny, cudaMemcpyDeviceToHost,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return MOSES_OK;
}

int moses_get_budget(moses_sim *s, double out[MOSES_BUDGET_LEN])
{
    if (!s || !out) return MOSES_EINVAL;
    const long long n = (long long)s->nx * (s->own_j1 - s->own_j0);  // the owned rows
    CK(cudaMemsetAsync(s->red, 0, 6 * sizeof(double), s->stream));
    if (s->prec == MOSES_FP64)
        budget_kernel<double><<<grid_for(n), 256, 0, s->stream>>>((const double *)s->U, nullptr, s->nx, s->own_j0,
                                                                  s->own_j1, s->pitch, s->plane, s->red);
    else
        budget_kernel<float><<<grid_for(n), 256, 0, s->stream>>>((const float *)s->U, rem<float>(s, s->U), s->nx,
                                                                 s->own_j0, s->own_j1, s->pitch, s->plane, s->red);
    CK(cudaGetLastError());
    double sums[6];
    CK(cudaMemcpyAsync(sums, s->red, sizeof(sums), cudaMemcpyDeviceToHost, s->stream));
    Ctl h;
    int rc = read_ctl(s, &h);
    if (rc) return rc;
    const double a = s->dx * s->dy;
    out[0] = sums[0] * a;
    out[1] = sums[3] * a;
    out[2] = sums[1] * a;
    out[3] = sums[2] * a;
    out[4] = sums[4] * a;
    out[5] = sums[5] * a;
    out[6] = h.bnd_in[0];
    out[7] = h.bnd_in[1];
    out[8] = h.clamp_vol[0];
    out[9] = h.clamp_vol[1];
    out[10] = (double)h.clamp_cells;
    out[11] = h.t;
    out[12] = (double)h.steps;
    return MOSES_OK;
}

// ---------------------------------------------------------------------------
// No-allocation step (moses_step_static).  Some callers cannot let a library
// call cudaMalloc: hosts that pre-reserve all device memory in their own pool
// (a foreign allocation fails or fragments it), processes that run under a
// hard device-memory limit, and loops that may not stall on the allocator
// (cudaMalloc and cudaFree synchronise the device).  For them, one FP64 Heun
// step of a small grid runs with all of its scratch (extended DEM, geometry
// planes, padded state, Heun intermediate, control block) in the statically
// sized device array below, which every GPU that loads this library holds
// until exit.  Every call shares the array: calls that overlap on the GPU race.

namespace {

constexpr int kStaticPitch = ((MOSES_STATIC_MAX_NX + 2 * GH) + 31) / 32 * 32;
constexpr long long kStaticPlane = (long long)kStaticPitch * (MOSES_STATIC_MAX_NY + 2 * GH);
constexpr long long kStaticCtl = 64;  // doubles reserved for the control block
constexpr long long kStaticDem = ((long long)(MOSES_STATIC_MAX_NX + 6) * (MOSES_STATIC_MAX_NY + 6) + 31) / 32 * 32;
constexpr long long kStaticDoubles = kStaticCtl + kStaticDem + (long long)(GEO_PLANES + 12) * kStaticPlane;
static_assert(sizeof(Ctl) <= kStaticCtl * sizeof(double), "control block does not fit");

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

// this process's device address of each device's copy of the array, looked up
// once per device (atomics: two host threads making a first call on the same
// device both look it up and store the same value)
std::atomic<double *> g_static_ptr[64];

__global__ void static_ctl_init_kernel(Ctl *ctl, double t)
{
    *ctl = Ctl{};
    ctl->t = t;
}

}  // namespace

int moses_step_static(const double *dem_device, int nx, int ny, double dx, double dy, const moses_params *p,
                      const double *U_in_device, double *U_out_device, double t, double *dt_out, void *stream)
{
    moses_sim *s = nullptr;  // errors of this call go to moses_last_error(NULL)
    if (!dem_device || !p || !U_in_device || !U_out_device) return fail(s, MOSES_EINVAL, "NULL argument");
    if (nx < 1 || ny < 1 || nx > MOSES_STATIC_MAX_NX || ny > MOSES_STATIC_MAX_NY)
        return fail(s, MOSES_EINVAL, "moses_step_static: grid must be 1..128 x 1..128 cells (static scratch limit)");
    if (!(std::isfinite(dx) && std::isfinite(dy) && dx > 0 && dy > 0) || !std::isfinite(t))
        return fail(s, MOSES_EINVAL, "dx, dy must be finite and > 0, t finite");
    std::string why;
    if (check_params(p, why)) return fail(s, MOSES_EINVAL, why);
    if (p->precision != MOSES_FP64) return fail(s, MOSES_EINVAL, "moses_step_static runs the FP64 form only");
    if (p->nu_f != 0.0) return fail(s, MOSES_EINVAL, "moses_step_static: nu_f must be 0");
    if (p->scheme != MOSES_SCHEME_CENTRAL || p->recon != MOSES_RECON_MINMOD || p->rk == 3 || p->k_mode != 0)
        return fail(s, MOSES_EINVAL, "moses_step_static: the paper's scheme only (scheme 0, recon 0, rk 2, k_mode 0)");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(s, MOSES_EINVAL, "device ordinal out of range");
    double *base = g_static_ptr[dev].load(std::memory_order_acquire);
    if (!base) {
        // host code may not use the array's name as a device address: ask the
        // runtime for this device's copy (first call per device; do it before
        // any stream capture)
        void *ptr = nullptr;
        CK(cudaGetSymbolAddress(&ptr, g_static_scratch));
        base = (double *)ptr;
        g_static_ptr[dev].store(base, std::memory_order_release);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int pitch = ((nx + 2 * GH) + 31) / 32 * 32;
    const long long plane = (long long)pitch * (ny + 2 * GH);
    Ctl *ctl = (Ctl *)base;
    double *bext = base + kStaticCtl;
    double *geo = bext + kStaticDem;
    double *U = geo + GEO_PLANES * plane;
    double *Us = U + 6 * plane;
    const long long n = (long long)nx * ny;
    // everything read below is written first except the unused tile corners:
    // clear the state planes so that stale data of earlier calls never enters
    CK(cudaMemsetAsync(U, 0, sizeof(double) * 12 * plane, st));
    static_ctl_init_kernel<<<1, 1, 0, st>>>(ctl, t);
    extend_dem_kernel<<<grid_for((long long)(nx + 6) * (ny + 6)), 256, 0, st>>>(dem_device, nx, ny, bext);
    const Phys phs = make_phys(p, dx, dy);
    geometry_kernel<double><<<grid_for((long long)(nx + 4) * (ny + 4)), 256, 0, st>>>(bext, nx, ny, pitch, plane, dx,
                                                                                     dy, phs, geo, 0);
    unpack_kernel<double><<<grid_for(6 * n), 256, 0, st>>>(U_in_device, U, nullptr, nx, ny, pitch, plane);
    CK(cudaGetLastError());
    StageArgs<double> a{};
    a.geo = geo;
    a.ctl = ctl;
    a.inflow = nullptr;
    a.n_inflow = 0;
    a.nx = nx;
    a.ny = ny;
    a.own_j0 = 0;
    a.own_j1 = ny;
    a.pitch = pitch;
    a.plane = plane;
    a.ph = phs;
    a.k = make_kt<double>(phs);
    fill_ghosts_kernel<double><<<grid_for(n), 256, 0, st>>>(a, U, t);
    max_speed_kernel<double><<<grid_for(n), 256, 0, st>>>(U, geo, nx, 0, ny, pitch, plane, &ctl->amax);
    CK(cudaGetLastError());
    StageArgs<double> a1 = a, a2 = a;
    a1.Uin = U;
    a1.Uout = Us;
    a1.stage = 1;
    a2.Uin = Us;
    a2.Un = U;
    a2.Uout = U;
    a2.stage = 2;
    a2.want_amax = 1;
    if (launch_stage<double>(a1, 0, st) || launch_stage<double>(a2, 0, st))
        return fail(s, MOSES_ECUDA, std::string("stage launch: ") + cudaGetErrorString(cudaGetLastError()));
    pack_kernel<double><<<grid_for(6 * n), 256, 0, st>>>(U, nullptr, U_out_device, nx, ny, pitch, plane);
    CK(cudaGetLastError());
    if (dt_out) {
        // the time step and the status word the stage kernels raise (a
        // non-finite value in the input or the result) in one copy
        Ctl h;
        CK(cudaMemcpyAsync(&h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *dt_out = h.dt;
        if (h.status & STATUS_TIMEOUT) return fail(s, MOSES_ETIMEOUT, "moses_step_static: a bounded device-side wait gave up");
        if (h.status & STATUS_NONFINITE)
            return fail(s, MOSES_ENONFINITE, "moses_step_static: the state or the time step became non-finite");
    }
    return MOSES_OK;
}

// ---------------------------------------------------------------------------
// Ensembles: many independent simulations (own DEM, parameters, grid size,
// time step) advanced together.  One cooperative launch runs every stage of
// every member for all the steps of a call (batch_persistent_kernel); the
// tile height is the fastest of 32 x 4, 32 x 8 and 32 x 16 on the members'
// own states, timed when the batch is made.  Members stay ordinary moses_sim
// objects.

struct moses_batch {
    int n = 0;
    int prec = MOSES_FP64;
    cudaStream_t stream = nullptr;       // the batch's own stream
    cudaStream_t user_stream = nullptr;  // the members' stream
    cudaEvent_t ev = nullptr;
    std::vector<moses_sim *> sims;
    void *args1 = nullptr, *args2 = nullptr;  // StageArgs<T>[n] for stage 1 / 2
    BatchStrip *strips = nullptr;  // (member, 32 x kStripRows strip) of every member
    int nstrips = 0;
    int ty = 8;                    // tile height of the launch
    int ntiles = 0;                // 32 x ty tiles of all members
    int cap = 0;                   // 32 x 4 tiles of all members (the most of any shape)
    int *tile_sim = nullptr;       // [cap] member of each tile
    int *tile_base = nullptr;      // [n] first tile of each member
    BatchTile *list = nullptr;     // wet-tile list (capacity cap)
    unsigned int *list_n = nullptr;
    unsigned char *zk = nullptr;   // known-zero flags of U* then U, [2][cap]
    unsigned short *mb = nullptr;  // mass bits of U then U*, [2][cap]
    GridSync *sync = nullptr;
    int *from_data = nullptr;
    int grid = 0;                  // CTAs of the launch
    int dbg_stall = 0;             // moses_batch_debug_timeout
    double tune_ms[3] = {0, 0, 0}; // one first stage per tile shape (32 x 4, 32 x 8, 32 x 16)
    Ctl **ctls = nullptr;
    Ctl *ctl_save = nullptr;       // the members' control blocks while the shapes are timed
    int *status = nullptr;
    std::string err;
};

namespace {

__global__ void batch_status_kernel(Ctl *const *ctls, int n, int *out)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        ctls[k]->dt_fixed = 0.0;
        ctls[k]->t_end = 0.0;
        if (ctls[k]->status) atomicOr(out, ctls[k]->status);
    }
}

__global__ void batch_ctl_copy_kernel(Ctl *const *ctls, Ctl *save, int n, int restore)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (restore) *ctls[k] = save[k];
        else save[k] = *ctls[k];
    }
}

int batch_fail(moses_batch *b, int code, const std::string &msg)
{
    if (b) b->err = msg;
    else g_create_err = msg;
    return code;
}

// the stage descriptors and the tile enumeration of the 32 x ty shape
template <typename T>
int batch_layout(moses_batch *b, int ty)
{
    std::vector<StageArgs<T>> a1(b->n), a2(b->n);
    std::vector<int> tile_sim, tile_base(b->n);
    for (int k = 0; k < b->n; k++) {
        moses_sim *s = b->sims[k];
        const int gx = (s->nx + 31) / 32, gy = (s->ny + ty - 1) / ty;
        tile_base[k] = (int)tile_sim.size();
        tile_sim.insert(tile_sim.end(), (size_t)gx * gy, k);
    }
    const size_t nt = tile_sim.size();
    for (int k = 0; k < b->n; k++) {
        moses_sim *s = b->sims[k];
        const size_t tb = (size_t)tile_base[k];
        a1[k] = base_args<T>(s);
        a1[k].Uin = (const T *)s->U;
        a1[k].Uout = (T *)s->Us;
        a1[k].Rin = rem<T>(s, s->U);
        a1[k].Rout = rem<T>(s, s->Us);
        a1[k].stage = 1;
        a2[k] = base_args<T>(s);
        a2[k].Uin = (const T *)s->Us;
        a2[k].Un = (const T *)s->U;
        a2[k].Uout = (T *)s->U;
        a2[k].Rin = rem<T>(s, s->Us);
        a2[k].Rn = rem<T>(s, s->U);
        a2[k].Rout = rem<T>(s, s->U);
        a2[k].stage = 2;
        a2[k].want_amax = 1;
        // the stage kernel runs listed tiles (the pointer marks it; the batch has its own list)
        a1[k].wl = a2[k].wl = s->wl;
        a1[k].zk = b->zk + tb;
        a2[k].zk = b->zk + b->cap + tb;
        a1[k].mb_in = b->mb + tb;
        a1[k].mb_out = b->mb + b->cap + tb;
        a2[k].mb_in = b->mb + b->cap + tb;
        a2[k].mb_n = b->mb + tb;
        a2[k].mb_out = b->mb + tb;
    }
    moses_sim *s = nullptr;  // CK reports into g_create_err
    CK(cudaMemcpyAsync(b->args1, a1.data(), sizeof(StageArgs<T>) * b->n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->args2, a2.data(), sizeof(StageArgs<T>) * b->n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->tile_sim, tile_sim.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->tile_base, tile_base.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));  // the host vectors go out of scope
    b->ty = ty;
    b->ntiles = (int)nt;
    return MOSES_OK;
}

// one launch of `nstages` stages; from_data: the first classifies from the data
template <typename T>
int batch_run(moses_batch *b, int nstages, bool from_data)
{
    moses_sim *s = nullptr;
    BatchRun<T> r{};
    r.args1 = (const StageArgs<T> *)b->args1;
    r.args2 = (const StageArgs<T> *)b->args2;
    r.nsim = b->n;
    r.strips = b->strips;
    r.nstrips = b->nstrips;
    r.tile_sim = b->tile_sim;
    r.tile_base = b->tile_base;
    r.ntiles = b->ntiles;
    r.list = b->list;
    r.list_n = b->list_n;
    r.sync = b->sync;
    r.from_data = b->from_data;
    r.nstages = 0;
    if (launch_batch<T>(r, b->ty, &b->grid, b->stream)) return batch_fail(b, MOSES_ECUDA, "ensemble kernel attributes");
    const GridSync g0{0u, 0u, (unsigned int)b->grid + (b->dbg_stall ? 1u : 0u), 0};
    const int fd = from_data ? 1 : 0;
    CK(cudaMemcpyAsync(b->sync, &g0, sizeof(GridSync), cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->from_data, &fd, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemsetAsync(b->list_n, 0, 2 * sizeof(unsigned int), b->stream));
    if (from_data) CK(cudaMemsetAsync(b->zk, 0, 2 * (size_t)b->cap, b->stream));
    r.nstages = nstages;
    if (nstages > 0 && launch_batch<T>(r, b->ty, nullptr, b->stream))
        return batch_fail(b, MOSES_ECUDA, std::string("ensemble launch: ") + cudaGetErrorString(cudaGetLastError()));
    return MOSES_OK;
}

// the tile height: one first stage per shape on the members' states (after
// one untimed first stage that classifies from the data), the fastest kept;
// the members' control blocks are restored afterwards (the stage writes U*,
// scratch between steps, and the time step and budgets in the control block)
template <typename T>
int batch_tune(moses_batch *b)
{
    moses_sim *s = nullptr;
    batch_ctl_copy_kernel<<<(b->n + 255) / 256, 256, 0, b->stream>>>(b->ctls, b->ctl_save, b->n, 0);
    CK(cudaGetLastError());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int shapes[3] = {4, 8, 16};
    int best = 8;
    double best_ms = 0.0;
    int rc = MOSES_OK;
    for (int q = 0; q < 3 && rc == MOSES_OK; q++) {
        rc = batch_layout<T>(b, shapes[q]);
        if (rc == MOSES_OK) rc = batch_run<T>(b, 1, true);
        float m = 0.f;
        if (rc == MOSES_OK) {
            cudaEventRecord(e0, b->stream);
            rc = batch_run<T>(b, 1, false);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&m, e0, e1) != cudaSuccess)
                rc = batch_fail(b, MOSES_ECUDA, "ensemble tile timing");
        }
        b->tune_ms[q] = m;
        if (rc == MOSES_OK && (q == 0 || m < best_ms)) {
            best = shapes[q];
            best_ms = m;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    batch_ctl_copy_kernel<<<(b->n + 255) / 256, 256, 0, b->stream>>>(b->ctls, b->ctl_save, b->n, 1);
    if (rc) return rc;
    CK(cudaGetLastError());
    GridSync g{};
    CK(cudaMemcpyAsync(&g, b->sync, sizeof(GridSync), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if (g.fail) return batch_fail(b, MOSES_ETIMEOUT, "a bounded device-side wait gave up while timing the tiles");
    return batch_layout<T>(b, best);
}

template <typename T>
int batch_build(moses_batch *b)
{
    std::vector<BatchStrip> strips;
    std::vector<Ctl *> ctls(b->n);
    long long cap = 0;
    for (int k = 0; k < b->n; k++) {
        moses_sim *s = b->sims[k];
        const int gx = (s->nx + 31) / 32;
        cap += (long long)gx * ((s->ny + 3) / 4);
        for (int sy = 0; sy < (s->ny + kStripRows - 1) / kStripRows; sy++)
            for (int sx = 0; sx < gx; sx++) strips.push_back(BatchStrip{k, sx, sy});
        ctls[k] = s->ctl;
    }
    if (cap > (1ll << 30)) return batch_fail(b, MOSES_EINVAL, "too many tiles in the batch");
    b->cap = (int)cap;
    b->nstrips = (int)strips.size();
    moses_sim *s = nullptr;  // CK reports into g_create_err
    CK(cudaMalloc(&b->args1, sizeof(StageArgs<T>) * b->n));
    CK(cudaMalloc(&b->args2, sizeof(StageArgs<T>) * b->n));
    CK(cudaMalloc(&b->strips, sizeof(BatchStrip) * strips.size()));
    CK(cudaMalloc(&b->list, sizeof(BatchTile) * (size_t)b->cap));
    CK(cudaMalloc(&b->list_n, 2 * sizeof(unsigned int)));
    CK(cudaMalloc(&b->tile_sim, sizeof(int) * (size_t)b->cap));
    CK(cudaMalloc(&b->tile_base, sizeof(int) * b->n));
    CK(cudaMalloc(&b->zk, 2 * (size_t)b->cap));
    CK(cudaMalloc(&b->mb, 2 * sizeof(unsigned short) * (size_t)b->cap));
    CK(cudaMalloc(&b->sync, sizeof(GridSync)));
    CK(cudaMalloc(&b->from_data, sizeof(int)));
    CK(cudaMalloc(&b->ctls, sizeof(Ctl *) * b->n));
    CK(cudaMalloc(&b->ctl_save, sizeof(Ctl) * b->n));
    CK(cudaMalloc(&b->status, sizeof(int)));
    CK(cudaMemcpyAsync(b->strips, strips.data(), sizeof(BatchStrip) * strips.size(), cudaMemcpyHostToDevice,
                       b->stream));
    CK(cudaMemcpyAsync(b->ctls, ctls.data(), sizeof(Ctl *) * b->n, cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return batch_tune<T>(b);
}

void free_batch(moses_batch *b)
{
    if (!b) return;
    cudaFree(b->args1);
    cudaFree(b->args2);
    cudaFree(b->strips);
    cudaFree(b->list);
    cudaFree(b->list_n);
    cudaFree(b->tile_sim);
    cudaFree(b->tile_base);
    cudaFree(b->zk);
    cudaFree(b->mb);
    cudaFree(b->sync);
    cudaFree(b->from_data);
    cudaFree(b->ctls);
    cudaFree(b->ctl_save);
    cudaFree(b->status);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}
}  // namespace

int moses_batch_create(int n, moses_sim *const *sims, moses_batch **out)
{
    if (!out) return batch_fail(nullptr, MOSES_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !sims) return batch_fail(nullptr, MOSES_EINVAL, "need n >= 1 simulations");
    for (int k = 0; k < n; k++) {
        if (!sims[k]) return batch_fail(nullptr, MOSES_EINVAL, "NULL simulation in the batch");
        if (sims[k]->prec != sims[0]->prec) return batch_fail(nullptr, MOSES_EINVAL, "members must share the precision");
        if (sims[k]->stream != sims[0]->stream) return batch_fail(nullptr, MOSES_EINVAL, "members must share the stream");
        if (!sims[k]->have_state) return batch_fail(nullptr, MOSES_ESTATE, "member without a state");
        if (sims[k]->p.nu_f != 0.0) return batch_fail(nullptr, MOSES_EINVAL, "members must have nu_f = 0");
        if (sims[k]->p.scheme != MOSES_SCHEME_CENTRAL || sims[k]->ph.recon != 0 || sims[k]->ph.rk != 2 ||
            sims[k]->ph.k_mode != 0)
            return batch_fail(nullptr, MOSES_EINVAL,
                              "members must use the paper's scheme (central, minmod, two-step, k_mode 0)");
        if (is_strip(sims[k])) return batch_fail(nullptr, MOSES_EINVAL, "a strip of a decomposed domain (owned rows set)");
        for (int q = 0; q < k; q++)
            if (sims[q] == sims[k]) return batch_fail(nullptr, MOSES_EINVAL, "a simulation appears twice");
    }
    moses_batch *b = new (std::nothrow) moses_batch();
    if (!b) return batch_fail(nullptr, MOSES_ENOMEM, "host allocation failed");
    b->n = n;
    b->prec = sims[0]->prec;
    b->user_stream = sims[0]->stream;
    b->sims.assign(sims, sims + n);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(b->ev, b->user_stream) != cudaSuccess || cudaStreamWaitEvent(b->stream, b->ev, 0) != cudaSuccess) {
        g_create_err = "batch stream or event creation failed";
        free_batch(b);
        return MOSES_ECUDA;
    }
    for (moses_sim *m : b->sims) zk_reset(m);  // timing the tile shapes writes the members' U*
    const int rc = b->prec == MOSES_FP64 ? batch_build<double>(b) : batch_build<float>(b);
    if (rc) {
        if (b->err.empty()) b->err = g_create_err;
        g_create_err = b->err;
        free_batch(b);
        return rc;
    }
    *out = b;
    return MOSES_OK;
}

static int batch_step(moses_batch *b, int nsteps, double *ms);

int moses_batch_step(moses_batch *b, int nsteps) { return batch_step(b, nsteps, nullptr); }

int moses_batch_step_timed(moses_batch *b, int nsteps, double *ms)
{
    if (!ms) return batch_fail(b, MOSES_EINVAL, "ms is NULL");
    return batch_step(b, nsteps, ms);
}

static int batch_step(moses_batch *b, int nsteps, double *ms)
{
    if (!b) return MOSES_EINVAL;
    if (nsteps < 0) return batch_fail(b, MOSES_EINVAL, "nsteps must be >= 0");
    for (moses_sim *m : b->sims) zk_reset(m);  // the batched launches write the members' buffers
    moses_sim *s = nullptr;
    // order after the members' pending work
    CK(cudaEventRecord(b->ev, b->user_stream));
    CK(cudaStreamWaitEvent(b->stream, b->ev, 0));
    CK(cudaMemsetAsync(b->status, 0, sizeof(int), b->stream));
    batch_status_kernel<<<(b->n + 255) / 256, 256, 0, b->stream>>>(b->ctls, b->n, b->status);  // CFL mode
    CK(cudaGetLastError());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, b->stream));
    }
    if (nsteps > 0) {
        const int rc = b->prec == MOSES_FP64 ? batch_run<double>(b, 2 * nsteps, true) : batch_run<float>(b, 2 * nsteps, true);
        if (rc) return rc;
    }
    if (ms) {
        CK(cudaEventRecord(e1, b->stream));
        CK(cudaEventSynchronize(e1));
        float m = 0.f;
        CK(cudaEventElapsedTime(&m, e0, e1));
        *ms = m;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    CK(cudaMemsetAsync(b->status, 0, sizeof(int), b->stream));
    batch_status_kernel<<<(b->n + 255) / 256, 256, 0, b->stream>>>(b->ctls, b->n, b->status);
    int st = 0;
    GridSync g{};
    CK(cudaMemcpyAsync(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(&g, b->sync, sizeof(GridSync), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    if (nsteps > 0 && g.fail) return batch_fail(b, MOSES_ETIMEOUT, "a bounded wait of the ensemble launch gave up");
    if (st & STATUS_TIMEOUT) return batch_fail(b, MOSES_ETIMEOUT, "a bounded device-side wait gave up");
    if (st & STATUS_NONFINITE) return batch_fail(b, MOSES_ENONFINITE, "a member became non-finite");
    return MOSES_OK;
}

int moses_batch_tiles(const moses_batch *b) { return b ? b->ntiles : 0; }

int moses_batch_tile_rows(const moses_batch *b, double ms_out[3])
{
    if (!b) return 0;
    if (ms_out)
        for (int q = 0; q < 3; q++) ms_out[q] = b->tune_ms[q];
    return b->ty;
}

int moses_batch_set_tile_rows(moses_batch *b, int rows)
{
    if (!b) return MOSES_EINVAL;
    if (rows != 4 && rows != 8 && rows != 16) return batch_fail(b, MOSES_EINVAL, "tile rows must be 4, 8 or 16");
    return b->prec == MOSES_FP64 ? batch_layout<double>(b, rows) : batch_layout<float>(b, rows);
}

int moses_batch_debug_timeout(moses_batch *b, int on)
{
    if (!b) return MOSES_EINVAL;
    b->dbg_stall = on ? 1 : 0;
    return MOSES_OK;
}

const char *moses_batch_last_error(const moses_batch *b) { return b ? b->err.c_str() : g_create_err.c_str(); }

void moses_batch_destroy(moses_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_batch(b);
}

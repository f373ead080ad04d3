// flux_eval.cu -- evaluation of a double-float flux phase
// (moses_debug_flux_eval): the stage's central flux through one face
// (face_flux2, twice the flux of Sect. 2.2 with the App. A fluxes) on
// synthetic faces, in FP64 and in double-float arithmetic (df64.cuh), timed
// and compared.  No stepping launch uses the double-float form.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/moses.h"
#include "internal.cuh"
#include "stage.cuh"
// after stage.cuh: the stage's own calls of fma on doubles are bound before
// the double-float fma is declared; its templates find the double-float
// overloads by argument-dependent lookup when instantiated on df
#include "df64.cuh"

using namespace moses;

namespace {

// splitmix64 (Steele, Lea and Flood 2014): a counter-based generator, so
// that every thread draws its face's numbers from the face index alone
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double unif(long long k, int c)  // [0, 1)
{
    return (double)(mix64((unsigned long long)k * 64ull + (unsigned long long)c) >> 11) * 0x1p-53;
}

// The two reconstructed states and the geometry of face k, of the magnitudes
// of a release event: per side and phase a mass J h of 0.05 .. 5 m (one in
// eight below J h_dry = 1e-4 m, with zero momenta, as the dry rule leaves
// them), velocities of -10 .. 10 m/s; the pressure coefficients of a bed
// sloped up to about 40 degrees.
__device__ void eval_face(long long k, double um[6], double up[6], FaceGeo<double> &G)
{
    G.jhd = 1e-4;
    G.sn = 0.5 + 4.5 * unif(k, 0);
    G.st = -0.5 + unif(k, 1);
    G.fn = 2.0 + 8.0 * unif(k, 2);
    G.ft = -1.0 + 2.0 * unif(k, 3);
    G.fn2 = 2.0 * G.fn;
    G.hg = 4.0 + unif(k, 4);
    double *side[2] = {um, up};
#pragma unroll
    for (int s = 0; s < 2; s++)
#pragma unroll
        for (int p = 0; p < 2; p++) {
            const int c0 = 8 + 8 * s + 4 * p;
            const bool dry = unif(k, c0) < 0.125;
            const double m = dry ? 0.9e-4 * unif(k, c0 + 1) : 0.05 + 4.95 * unif(k, c0 + 1);
            side[s][3 * p] = m;
            side[s][3 * p + 1] = dry ? 0.0 : m * (-10.0 + 20.0 * unif(k, c0 + 2));
            side[s][3 * p + 2] = dry ? 0.0 : m * (-10.0 + 20.0 * unif(k, c0 + 3));
        }
}

// A face's inputs: um[6], up[6] and the seven geometry terms, 19 values,
// stored as 19 planes of n elements of the arithmetic type
constexpr int kFaceIn = 19;

__device__ __forceinline__ void put(double *p, long long i, double x) { p[i] = x; }
__device__ __forceinline__ void put(df *p, long long i, double x) { p[i] = df(x); }
__device__ __forceinline__ double as_double(double x) { return x; }
__device__ __forceinline__ double as_double(df x) { return x.to_double(); }

// the faces' inputs in both types (untimed: the conversions to double-float
// run here, on the FP64 pipe, and not in the timed kernels)
__global__ void flux_eval_setup_kernel(long long n, double *in64, df *indf)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += stride) {
        double v[kFaceIn];
        FaceGeo<double> G;
        eval_face(k, v, v + 6, G);
        v[12] = G.jhd;
        v[13] = G.sn;
        v[14] = G.st;
        v[15] = G.fn;
        v[16] = G.ft;
        v[17] = G.fn2;
        v[18] = G.hg;
#pragma unroll
        for (int c = 0; c < kFaceIn; c++) {
            put(in64, c * n + k, v[c]);
            put(indf, c * n + k, v[c]);
        }
    }
}

// the next repetition's input depends on this one's output, times a zero the
// compiler cannot see: no repetition is hoisted or dropped, no value changes
__device__ __forceinline__ void feed(double &u, double h, double zd, float) { u = ::fma(zd, h, u); }
__device__ __forceinline__ void feed(df &u, df h, double, float zf) { u.hi = fmaf(zf, h.hi, u.hi); }

// in: kFaceIn planes of n; out: 7 planes of n, the fluxes of the last
// repetition, both in the arithmetic type (no conversion in the timed kernel)
template <typename T>
__global__ void __launch_bounds__(256) flux_eval_kernel(long long n, int reps, double zd, float zf, const T *in, T *out)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += stride) {
        T um[6], up[6];
#pragma unroll
        for (int c = 0; c < 6; c++) {
            um[c] = in[c * n + k];
            up[c] = in[(6 + c) * n + k];
        }
        const FaceGeo<T> G{in[12 * n + k], in[13 * n + k], in[14 * n + k], in[15 * n + k],
                           in[16 * n + k], in[17 * n + k], in[18 * n + k]};
        T H[7];
        for (int r = 0; r < reps; r++) {
            face_flux2<T, 0>(um, up, G, G, H);
#pragma unroll
            for (int c = 0; c < 6; c++) feed(um[c], H[c], zd, zf);
            feed(up[0], H[6], zd, zf);
        }
#pragma unroll
        for (int c = 0; c < 7; c++) out[c * n + k] = H[c];
    }
}

// the double-float fluxes as doubles (untimed)
__global__ void flux_eval_widen_kernel(long long m, const df *a, double *b)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m; k += stride) b[k] = as_double(a[k]);
}

__device__ __forceinline__ void max_bits(double *dst, double v)  // v >= 0
{
    atomicMax(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)__double_as_longlong(v));
}

// acc[c] = max |a_c|, acc[7 + c] = max |b_c - a_c| over the n faces
__global__ void flux_diff_kernel(long long n, const double *a, const double *b, double *acc)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    double ma[7] = {}, md[7] = {};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += stride)
#pragma unroll
        for (int c = 0; c < 7; c++) {
            ma[c] = fmax(ma[c], fabs(a[c * n + k]));
            md[c] = fmax(md[c], fabs(b[c * n + k] - a[c * n + k]));
        }
#pragma unroll
    for (int c = 0; c < 7; c++) {
        max_bits(acc + c, ma[c]);
        max_bits(acc + 7 + c, md[c]);
    }
}

// acc[14] = max |b - a| / |a| over the components with |a| > 1e-6 of the
// component's largest |a| (acc[0..6])
__global__ void flux_rel_kernel(long long n, const double *a, const double *b, double *acc)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    double m = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += stride)
#pragma unroll
        for (int c = 0; c < 7; c++) {
            const double x = fabs(a[c * n + k]);
            if (x > 1e-6 * acc[c]) m = fmax(m, fabs(b[c * n + k] - a[c * n + k]) / x);
        }
    max_bits(acc + 14, m);
}

}  // namespace

int moses_debug_flux_eval(long long n, int reps, double *res)
{
    moses_sim *s = nullptr;  // errors go to moses_last_error(NULL)
    if (!res || n < 1 || n > (1ll << 22) || reps < 4 || reps > 64)
        return fail(s, MOSES_EINVAL, "need res, 1 <= n <= 2^22 and 4 <= reps <= 64");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // inputs (19 planes) and fluxes (7 planes) of both types, the double-float
    // fluxes widened to doubles, the reduction words
    unsigned char *d = nullptr;
    const size_t plane8 = sizeof(double) * (size_t)n;
    CK(cudaMalloc(&d, plane8 * (2 * kFaceIn + 2 * 7 + 7) + sizeof(double) * 16));
    double *in64 = reinterpret_cast<double *>(d);
    df *indf = reinterpret_cast<df *>(d + plane8 * kFaceIn);
    double *out64 = reinterpret_cast<double *>(d + plane8 * 2 * kFaceIn);
    df *outdf = reinterpret_cast<df *>(d + plane8 * (2 * kFaceIn + 7));
    double *wide = reinterpret_cast<double *>(d + plane8 * (2 * kFaceIn + 14));
    double *acc = reinterpret_cast<double *>(d + plane8 * (2 * kFaceIn + 21));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = sms * 8, threads = 256;
    if (e == cudaSuccess) {
        flux_eval_setup_kernel<<<blocks, threads>>>(n, in64, indf);
        e = cudaGetLastError();
    }
    // the fastest of three launches of `r` repetitions
    const auto timed = [&](bool dbl, int r) -> double {
        float best = 1e30f;
        for (int t = 0; t < 3 && e == cudaSuccess; t++) {
            cudaEventRecord(e0);
            if (dbl) flux_eval_kernel<double><<<blocks, threads>>>(n, r, 0.0, 0.0f, in64, out64);
            else flux_eval_kernel<df><<<blocks, threads>>>(n, r, 0.0, 0.0f, indf, outdf);
            cudaEventRecord(e1);
            e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        return (double)best;
    };
    // the flux alone: the difference of `reps` and 2 repetitions (the loads
    // and the stores cancel); the `reps` launches run last, so that both
    // output buffers hold their results
    const double t64_2 = timed(true, 2);
    const double t64 = timed(true, reps) - t64_2;
    const double tdf_2 = timed(false, 2);
    const double tdf = timed(false, reps) - tdf_2;
    double h[15] = {};
    if (e == cudaSuccess) e = cudaMemset(acc, 0, sizeof(double) * 16);
    if (e == cudaSuccess) {
        flux_eval_widen_kernel<<<blocks, threads>>>(7 * n, outdf, wide);
        flux_diff_kernel<<<blocks, threads>>>(n, out64, wide, acc);
        flux_rel_kernel<<<blocks, threads>>>(n, out64, wide, acc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, acc, sizeof(h), cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    if (e != cudaSuccess) return fail(s, MOSES_ECUDA, std::string("moses_debug_flux_eval: ") + cudaGetErrorString(e));
    const double faces = (double)n * (reps - 2);
    res[0] = t64 > 0.0 ? faces / (t64 * 1e-3) / 1e9 : 0.0;
    res[1] = tdf > 0.0 ? faces / (tdf * 1e-3) / 1e9 : 0.0;
    double norm = 0.0;
    for (int c = 0; c < 7; c++)
        if (h[c] > 0.0) norm = std::max(norm, h[7 + c] / h[c]);
    res[2] = norm;
    res[3] = h[14];
    return MOSES_OK;
}

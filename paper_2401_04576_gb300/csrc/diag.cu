// Directed-rounding pipe microbenchmark (roofline denominators for the ALU-bound vote
// kernels): independent dependency chains per thread, grid covering every SM.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace apo {

constexpr int kChains = 8;
constexpr int kIters = 2048;

__device__ __forceinline__ double dsqrt_lib(double x) { return __dsqrt_rd(x); }
__device__ __forceinline__ float dsqrt_lib(float x) { return __fsqrt_rd(x); }

template <typename T, int OP>
__global__ void __launch_bounds__(256) k_pipe(T seed, T *sink) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = seed + T(c) * T(1e-3) + T(threadIdx.x) * T(1e-6);
    const T a = T(1e-7), m = T(0.9999999);
#pragma unroll 4
    for (int i = 0; i < kIters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
            if (OP == 0) x[c] = rd_add(x[c], a);
            else if (OP == 1) x[c] = rd_mul(x[c], m);
            else if (OP == 2) x[c] = (i & 1) ? rd_mul(x[c], m) : ru_add(x[c], a);
            else if (OP == 3) x[c] = (i & 1) ? rd_mul(x[c], T(3)) : rd_sqrt(x[c]);
            else x[c] = (i & 1) ? rd_mul(x[c], T(3)) : dsqrt_lib(x[c]);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    if (s == T(-12345)) *sink = s;   // keeps the chains alive
}

template <typename T, int OP> static double run_pipe() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    T *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return -1.0;
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_pipe<T, OP><<<blocks, threads>>>(T(1), sink);   // warm-up
    cudaEventRecord(e0);
    const int reps = 3;
    for (int r = 0; r < reps; r++) k_pipe<T, OP><<<blocks, threads>>>(T(1), sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1.0;
    double ops = (double)reps * blocks * threads * kIters * kChains;
    return ops / (ms * 1e-3);
}

double pipe_peak(int precision, int op) {
    if (precision == 0) {
        if (op == 0) return run_pipe<double, 0>();
        if (op == 1) return run_pipe<double, 1>();
        if (op == 3) return run_pipe<double, 3>();
        if (op == 4) return run_pipe<double, 4>();
        return run_pipe<double, 2>();
    }
    if (op == 0) return run_pipe<float, 0>();
    if (op == 1) return run_pipe<float, 1>();
    return run_pipe<float, 2>();
}

// Elementwise scalar operations for the tests of ipipe.cuh.
// x has an even number of elements when op is a quotient (12-17).
__global__ void k_dops(int op, const double *__restrict__ x, double *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        double r;
        switch (op) {
            case 0: r = ipipe::rcp_rd(v); break;
            case 1: r = ipipe::rcp_ru(v); break;
            case 2: r = ipipe::rcp_rn(v); break;
            case 3: r = ipipe::sqrt_rd(v); break;
            case 4: r = ipipe::sqrt_ru(v); break;
            case 5: r = ipipe::sqrt_rn(v); break;
            case 6: r = __drcp_rd(v); break;
            case 7: r = __drcp_ru(v); break;
            case 8: r = __drcp_rn(v); break;
            case 9: r = __dsqrt_rd(v); break;
            case 10: r = __dsqrt_ru(v); break;
            case 11: r = __dsqrt_rn(v); break;
            // quotients x[i] / x[i ^ 1]
            case 12: r = ipipe::div_rd(v, x[i ^ 1]); break;
            case 13: r = ipipe::div_ru(v, x[i ^ 1]); break;
            case 14: r = ipipe::div_rn(v, x[i ^ 1]); break;
            case 15: r = __ddiv_rd(v, x[i ^ 1]); break;
            case 16: r = __ddiv_ru(v, x[i ^ 1]); break;
            default: r = __ddiv_rn(v, x[i ^ 1]); break;
        }
        out[i] = r;
    }
}

// The vote program's end points for explicit (cell, hit) pairs: cells as 12 doubles (D, sin
// phi0, cos phi0, omega, z0, tan(lambda), lo / hi each), hits as 9 doubles (x0, y0, sin
// phi_s, cos phi_s, tan tau, sin phi_s tan tau, cos phi_s tan tau, tan^2 tau, drift).  FP32
// rounds both outward, as the staging and the cell lookup do.  out: 10 doubles per pair,
// the vote then the 9 of vote_pair_ends.
__global__ void k_pair_ends(SeriesConsts k, int precision, const double *__restrict__ cells,
                            const double *__restrict__ hits, double *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double *c = cells + 12 * i, *h = hits + 9 * i;
        double *o = out + 10 * i;
        bool v;
        if (precision == 0) {
            Cell<double> cd{{c[0], c[1]}, {c[2], c[3]}, {c[4], c[5]}, {c[6], c[7]}, {c[8], c[9]}, {c[10], c[11]}};
            Hit<double> hd;
            IV<double> *f = &hd.x0;
            for (int j = 0; j < 9; j++) f[j] = {h[j], h[j]};
            v = vote_pair_ends<double>(cd, hd, k, o + 1);
        } else {
            Cell<float> cf;
            IV<float> *cc = &cf.D;
            for (int j = 0; j < 6; j++) cc[j] = {__double2float_rd(c[2 * j]), __double2float_ru(c[2 * j + 1])};
            Hit<float> hf;
            IV<float> *f = &hf.x0;
            for (int j = 0; j < 9; j++) f[j] = {__double2float_rd(h[j]), __double2float_ru(h[j])};
            v = vote_pair_ends<float>(cf, hf, k, o + 1);
        }
        o[0] = v ? 1.0 : 0.0;
    }
}

int launch_pair_ends(const SeriesConsts &k, int precision, const double *cells, const double *hits,
                     double *out, long long n, cudaStream_t s) {
    if (n <= 0) return 0;
    const long long want = (n + 127) / 128;
    const int blocks = (int)(want < 4096 ? want : 4096);
    k_pair_ends<<<blocks, 128, 0, s>>>(k, precision, cells, hits, out, n);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_dops(int op, const double *x, double *out, long long n, cudaStream_t s) {
    if (n <= 0) return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + 255) / 256;
    const int blocks = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    k_dops<<<blocks, 256, 0, s>>>(op, x, out, n);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace apo

// GPU helper of the builder: products of kernel blocks with tall, skinny
// matrices, Y = K(rows, cols) M, evaluated on the fly.  Used by the
// randomized SVD of large admissible blocks (Halko, Martinsson, Tropp
// 2011): Y = A Omega, the power iterations and B^T = A^T Q (the kernels are
// symmetric, so A^T is the block with rows and columns swapped).
//
// The kernel is evaluated in float from float coordinates and multiplied in
// float; every 128-column chunk's partial sum is added into a double
// accumulator.  Construction is outside the paper's scope (end of
// Section 2); this only speeds up building large H-matrices.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "hm_device.h"
#include "hm_internal.h"

namespace hm {
namespace {

constexpr int kRows = 128;   // rows (threads) per CTA
constexpr int kChunk = 128;  // columns staged per step

struct DevTask {
    int64_t row0, nrows, col0, ncols, m_off, y_off;
    int64_t tile0;  // first row tile of this task in the flattened grid
};

template <int ELL>
__global__ void __launch_bounds__(kRows) sketch_kernel(const DevTask* __restrict__ tasks, int ntasks,
                                                       const float* __restrict__ pts,
                                                       const int64_t* __restrict__ idx, int d,
                                                       int kernel, int ell,
                                                       const float* __restrict__ M,
                                                       double* __restrict__ Y, int* bad) {
    __shared__ float sp[kChunk * 3];
    __shared__ int64_t si[kChunk];
    __shared__ float sm[kChunk * ELL];
    // locate the task of this CTA (tasks sorted by tile0)
    int lo = 0, hi = ntasks - 1;
    const int64_t tile = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
    }
    const DevTask t = tasks[lo];
    const int64_t a = (tile - t.tile0) * kRows + threadIdx.x;
    const bool active = a < t.nrows;
    float px = 0.f, py = 0.f, pz = 0.f;
    int64_t ia = -1;
    if (active) {
        const int64_t p = t.row0 + a;
        px = pts[p * 3 + 0];
        py = pts[p * 3 + 1];
        pz = pts[p * 3 + 2];
        ia = idx[p];
    }
    double accd[ELL];
#pragma unroll
    for (int c = 0; c < ELL; ++c) accd[c] = 0.0;
    const float inv4pi = 0.0795774715459476679f;
    for (int64_t b0 = 0; b0 < t.ncols; b0 += kChunk) {
        const int nb = (int)((t.ncols - b0) < kChunk ? (t.ncols - b0) : kChunk);
        __syncthreads();
        for (int e = threadIdx.x; e < nb; e += kRows) {
            const int64_t q = t.col0 + b0 + e;
            sp[e * 3 + 0] = pts[q * 3 + 0];
            sp[e * 3 + 1] = pts[q * 3 + 1];
            sp[e * 3 + 2] = pts[q * 3 + 2];
            si[e] = idx[q];
        }
        for (int e = threadIdx.x; e < nb * ELL; e += kRows) {
            const int bb = e / ELL, c = e - bb * ELL;
            sm[e] = c < ell ? M[t.m_off + (b0 + bb) * ell + c] : 0.f;
        }
        __syncthreads();
        if (!active) continue;
        float acc[ELL];
#pragma unroll
        for (int c = 0; c < ELL; ++c) acc[c] = 0.f;
        for (int bb = 0; bb < nb; ++bb) {
            const float dx = px - sp[bb * 3 + 0];
            const float dy = py - sp[bb * 3 + 1];
            const float dz = pz - sp[bb * 3 + 2];
            const float r2 = dx * dx + dy * dy + dz * dz;
            float kv;
            if (si[bb] == ia) {
                kv = 1.f;
            } else if (r2 == 0.f) {
                atomicOr(bad, 1);
                kv = 0.f;
            } else if (kernel == HMAT_K_LOG2D) {
                kv = -0.5f * logf(r2);
            } else {
                kv = inv4pi * rsqrtf(r2);
            }
            const float* mrow = sm + bb * ELL;
#pragma unroll
            for (int c = 0; c < ELL; ++c) acc[c] = fmaf(kv, mrow[c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < ELL; ++c) accd[c] += (double)acc[c];
    }
    if (active) {
        double* yr = Y + t.y_off + a * ell;
#pragma unroll
        for (int c = 0; c < ELL; ++c)
            if (c < ell) yr[c] = accd[c];
    }
}

template <int ELL>
void launch_sketch(int64_t tiles, const DevTask* tasks, int ntasks, const float* pts,
                   const int64_t* idx, int d, int kernel, int ell, const float* M, double* Y,
                   int* bad, cudaStream_t st) {
    sketch_kernel<ELL><<<(unsigned)tiles, kRows, 0, st>>>(tasks, ntasks, pts, idx, d, kernel, ell,
                                                        M, Y, bad);
    count_launches(1);
}

}  // namespace

struct GpuSketch {
    int device = 0, d = 2, kernel = 0;
    int64_t N = 0;
    float* pts = nullptr;       // tree order, N x 3 (z = 0 in 2D)
    int64_t* idx = nullptr;     // original index of each tree position
    int* bad = nullptr;
    cudaStream_t st = nullptr;
};

#define SK_TRY(call)                                                                   \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            set_error("build sketch: %s: %s", #call, cudaGetErrorString(e_));          \
            return HMAT_ECUDA;                                                         \
        }                                                                              \
    } while (0)

int gpu_sketch_init(GpuSketch** out, int device, const double* pts_tree, const int64_t* orig,
                    int64_t N, int d, int kernel) {
    GpuSketch* s = new GpuSketch();
    *out = s;
    s->device = device;
    s->d = d;
    s->kernel = kernel;
    s->N = N;
    SK_TRY(cudaSetDevice(device));
    SK_TRY(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
    std::vector<float> p3((size_t)N * 3, 0.f);
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < d; ++k) p3[i * 3 + k] = (float)pts_tree[i * d + k];
    SK_TRY(cudaMalloc(&s->pts, p3.size() * sizeof(float)));
    SK_TRY(cudaMalloc(&s->idx, (size_t)N * sizeof(int64_t)));
    SK_TRY(cudaMalloc(&s->bad, sizeof(int)));
    SK_TRY(cudaMemcpy(s->pts, p3.data(), p3.size() * sizeof(float), cudaMemcpyHostToDevice));
    SK_TRY(cudaMemcpy(s->idx, orig, (size_t)N * sizeof(int64_t), cudaMemcpyHostToDevice));
    SK_TRY(cudaMemset(s->bad, 0, sizeof(int)));
    return HMAT_OK;
}

void gpu_sketch_free(GpuSketch* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->pts) cudaFree(s->pts);
    if (s->idx) cudaFree(s->idx);
    if (s->bad) cudaFree(s->bad);
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
}

int gpu_sketch_apply(GpuSketch* s, const std::vector<SketchTask>& tasks, int ell,
                     const std::vector<float>& M, std::vector<double>& Y) {
    if (tasks.empty()) return HMAT_OK;
    if (ell < 1 || ell > 64) {
        set_error("build sketch: sketch width %d outside 1..64", ell);
        return HMAT_EUNSUPPORTED;
    }
    SK_TRY(cudaSetDevice(s->device));
    std::vector<DevTask> dt(tasks.size());
    int64_t tiles = 0;
    for (size_t i = 0; i < tasks.size(); ++i) {
        const SketchTask& t = tasks[i];
        dt[i] = DevTask{t.row0, t.nrows, t.col0, t.ncols, t.m_off, t.y_off, tiles};
        tiles += (t.nrows + kRows - 1) / kRows;
    }
    DevTask* d_tasks = nullptr;
    float* d_M = nullptr;
    double* d_Y = nullptr;
    auto cleanup = [&]() {
        if (d_tasks) cudaFree(d_tasks);
        if (d_M) cudaFree(d_M);
        if (d_Y) cudaFree(d_Y);
    };
    cudaError_t e = cudaMalloc(&d_tasks, dt.size() * sizeof(DevTask));
    if (e == cudaSuccess) e = cudaMalloc(&d_M, M.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d_Y, Y.size() * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tasks, dt.data(), dt.size() * sizeof(DevTask), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_M, M.data(), M.size() * sizeof(float), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess && tiles > 0) {
        const int w = ell <= 8 ? 8 : ell <= 16 ? 16 : ell <= 24 ? 24 : ell <= 32 ? 32
                    : ell <= 40 ? 40 : ell <= 48 ? 48 : 64;
        const int nt = (int)dt.size();
        switch (w) {
            case 8: launch_sketch<8>(tiles, d_tasks, nt, s->pts, s->idx, s->d, s->kernel, ell, d_M, d_Y, s->bad, s->st); break;
            case 16: launch_sketch<16>(tiles, d_tasks, nt, s->pts, s->idx, s->d, s->kernel, ell, d_M, d_Y, s->bad, s->st); break;
            case 24: launch_sketch<24>(tiles, d_tasks, nt, s->pts, s->idx, s->d, s->kernel, ell, d_M, d_Y, s->bad, s->st); break;
            case 32: launch_sketch<32>(tiles, d_tasks, nt, s->pts, s->idx, s->d, s->kernel, ell, d_M, d_Y, s->bad, s->st); break;
            case 40: launch_sketch<40>(tiles, d_tasks, nt, s->pts, s->idx, s->d, s->kernel, ell, d_M, d_Y, s->bad, s->st); break;
            case 48: launch_sketch<48>(tiles, d_tasks, nt, s->pts, s->idx, s->d, s->kernel, ell, d_M, d_Y, s->bad, s->st); break;
            default: launch_sketch<64>(tiles, d_tasks, nt, s->pts, s->idx, s->d, s->kernel, ell, d_M, d_Y, s->bad, s->st); break;
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(Y.data(), d_Y, Y.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    int bad = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bad, s->bad, sizeof(int), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    cleanup();
    if (e != cudaSuccess) {
        set_error("build sketch: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? HMAT_ENOMEM : HMAT_ECUDA;
    }
    if (bad) {
        set_error("hmat_build: two distinct points coincide");
        return HMAT_EINVAL;
    }
    return HMAT_OK;
}

}  // namespace hm

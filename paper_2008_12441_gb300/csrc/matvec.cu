// CUDA-core kernels of the single-GPU H-matrix-vector product.
//
// The paper's distributed algorithm (Section 4.1) runs five steps; on one
// GPU they become two kernels over a padded, level-major layout:
//
//   project (Step 1, eq. (prod-vx)): for every low-rank level l and every
//     source node j, the s sibling products V_ij^T x_j at once, as s*r_l
//     dot products over the node's slots.  One CTA owns a tile of slots
//     across ALL levels (x is read once); nodes longer than the tile leave
//     one partial sum per tile.
//   expand (Steps 2-5, eqs. (prod-yuz), (prod-ydz)): every CTA first sums
//     the partials of the sibling nodes it needs, in a fixed order (Step 2's
//     tree reduction without atomics; Steps 3-4 are the index transpose
//     "slot of i at source j" and need no data movement), then streams its
//     rows of the dense near-field block and of every level's U factor and
//     writes each y element exactly once.
//
// Every accumulation order is fixed, so results are bitwise reproducible.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "hm_device.h"

namespace hm {
namespace {

template <typename A, int VEC>
struct VecLoad;

template <>
struct VecLoad<float, 4> {
    static __device__ __forceinline__ void go(const float* p, float (&o)[4]) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <>
struct VecLoad<float, 2> {
    static __device__ __forceinline__ void go(const float* p, float (&o)[2]) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
};
template <>
struct VecLoad<float, 1> {
    static __device__ __forceinline__ void go(const float* p, float (&o)[1]) { o[0] = __ldg(p); }
};
template <>
struct VecLoad<double, 2> {
    static __device__ __forceinline__ void go(const double* p, double (&o)[2]) {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
};
template <>
struct VecLoad<double, 1> {
    static __device__ __forceinline__ void go(const double* p, double (&o)[1]) { o[0] = __ldg(p); }
};

// ------------------------------------------------------------------ project
// grid: Np / tile_p CTAs, 256 threads.  smem: tile_p * KC values of x.
template <typename A, int KC, int VEC>
__global__ void __launch_bounds__(256) project_kernel(const MatvecArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    A* xs = reinterpret_cast<A*>(smem_raw);
    const int64_t tile = a.tile_p;
    const int64_t p0 = (int64_t)blockIdx.x * tile;
    const A* __restrict__ x = static_cast<const A*>(a.x);
    const A* __restrict__ V = static_cast<const A*>(a.V);

    for (int64_t e = threadIdx.x; e < tile * KC; e += blockDim.x) {
        const int64_t pl = e / KC;
        const int c = (int)(e - pl * KC);
        const int64_t src = a.map ? a.map[p0 + pl] : p0 + pl;
        xs[e] = (src >= 0 && c < a.k) ? x[src * a.ldx + c] : A(0);
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    for (int l = 1; l <= a.nf; ++l) {
        const DevLevel L = a.lv[l];
        const int sr = a.s * L.r;
        if (sr == 0) continue;
        const int64_t seg = L.seg_len;
        const int nseg_t = (int)(tile / seg);
        const int rows = nseg_t * sr;
        A* Tl = static_cast<A*>(a.T) + L.t_off * a.kc;
        for (int row = warp; row < rows; row += nw) {
            const int sg = row / sr;
            const int col = row - sg * sr;
            const int64_t ps = p0 + (int64_t)sg * seg;
            const int64_t node = ps / L.n;
            const A* v = V + L.fac_off + (node * sr + col) * L.n + (ps - node * L.n);
            const A* xl = xs + (int64_t)sg * seg * KC;
            A acc[KC];
#pragma unroll
            for (int c = 0; c < KC; ++c) acc[c] = A(0);
#pragma unroll 4
            for (int64_t i = (int64_t)lane * VEC; i < seg; i += 32 * VEC) {
                A vv[VEC];
                VecLoad<A, VEC>::go(v + i, vv);
#pragma unroll
                for (int e = 0; e < VEC; ++e)
#pragma unroll
                    for (int c = 0; c < KC; ++c) acc[c] += vv[e] * xl[(i + e) * KC + c];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int c = 0; c < KC; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
            A* dst = Tl + ((ps / seg) * sr + col) * a.kc;
#pragma unroll
            for (int c = 0; c < KC; ++c)
                if ((c & 31) == lane && c < a.k) dst[c] = acc[c];
        }
    }
}

// ------------------------------------------------------------------- expand
// grid: Np / tile_e CTAs, min(256, tile_e / VEC) threads, each looping over
// its VEC-slot groups of the tile.  smem: x of the near-field
// group(s) covering the tile, then per level the summed partial products
// t_{i<-j} of the tile's target nodes, [node][s*r_l][KC].
template <typename A, int KC, int VEC>
__global__ void __launch_bounds__(256) expand_kernel(const MatvecArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t TE = a.tile_e;
    const int64_t e0 = (int64_t)blockIdx.x * TE;
    const int64_t G = a.G;
    const int64_t gx0 = (e0 / G) * G;
    const int64_t GX = TE > G ? TE : G;
    const int nc = a.s + 1;
    const A* __restrict__ x = static_cast<const A*>(a.x);
    A* xg = reinterpret_cast<A*>(smem_raw);
    A* ttb = xg + GX * KC;

    for (int64_t e = threadIdx.x; e < GX * KC; e += blockDim.x) {
        const int64_t b = e / KC;
        const int c = (int)(e - b * KC);
        const int64_t slot = gx0 + b;
        const int64_t src = a.map ? a.map[slot] : slot;
        xg[e] = (src >= 0 && c < a.k) ? x[src * a.ldx + c] : A(0);
    }
    // Step 2 (+3, 4): fixed-order sum of the sibling partials each target
    // node of the tile needs; slot qv of target i at source j is the index
    // transpose of slot qp of source j at target i.
    int64_t ttoff[kMaxLevels + 1];
    {
        int64_t off = 0;
        for (int l = 1; l <= a.nf; ++l) {
            const DevLevel L = a.lv[l];
            const int sr = a.s * L.r;
            const int64_t nodes_t = TE >= L.n ? TE / L.n : 1;
            const int64_t i0 = e0 / L.n;
            const int64_t nsub = L.n / L.seg_len;
            const A* Tl = static_cast<const A*>(a.T) + L.t_off * a.kc;
            A* ttl = ttb + off;
            const int64_t total = nodes_t * sr * KC;
            for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
                const int c = (int)(e % KC);
                const int64_t rest = e / KC;
                const int col = (int)(rest % sr);
                const int64_t i = i0 + rest / sr;
                const int ci = (int)(i % nc);
                const int qp = col / L.r, cr = col - qp * L.r;
                const int cj = qp < ci ? qp : qp + 1;
                const int64_t j = i - ci + cj;
                const int qv = ci < cj ? ci : ci - 1;
                A sum = A(0);
                if (c < a.k)
                    for (int64_t u = 0; u < nsub; ++u)
                        sum += Tl[((j * nsub + u) * sr + qv * L.r + cr) * a.kc + c];
                ttl[e] = sum;
            }
            ttoff[l] = off;
            off += total;
        }
    }
    __syncthreads();

    const A* __restrict__ D = static_cast<const A*>(a.D);
    const A* __restrict__ U = static_cast<const A*>(a.U);
    A* __restrict__ y = static_cast<A*>(a.y);
    for (int64_t sv = e0 + (int64_t)threadIdx.x * VEC; sv < e0 + TE;
         sv += (int64_t)blockDim.x * VEC) {
        A acc[VEC][KC];
#pragma unroll
        for (int v = 0; v < VEC; ++v)
#pragma unroll
            for (int c = 0; c < KC; ++c) acc[v][c] = A(0);

        // Step 5, dense near-field block: y_p += sum_b D[p][b] x_b (eq. (prod-ydz))
        {
            const int64_t g = sv / G;
            const A* Dg = D + g * G * G + (sv - g * G);
            const A* xgg = xg + (g * G - gx0) * KC;
#pragma unroll 4
            for (int64_t b = 0; b < G; ++b) {
                A dv[VEC];
                VecLoad<A, VEC>::go(Dg + b * G, dv);
#pragma unroll
                for (int v = 0; v < VEC; ++v)
#pragma unroll
                    for (int c = 0; c < KC; ++c) acc[v][c] += dv[v] * xgg[b * KC + c];
            }
        }
        // Step 5, low-rank blocks, finest level first: y_p += U_p t (eq. (prod-yuz))
        for (int l = a.nf; l >= 1; --l) {
            const DevLevel L = a.lv[l];
            const int sr = a.s * L.r;
            const int64_t i = sv / L.n;
            const int64_t il = i - e0 / L.n;
            const A* u = U + L.fac_off + i * sr * L.n + (sv - i * L.n);
            const A* tl = ttb + ttoff[l] + il * sr * KC;
#pragma unroll 4
            for (int col = 0; col < sr; ++col) {
                A uv[VEC];
                VecLoad<A, VEC>::go(u + (int64_t)col * L.n, uv);
#pragma unroll
                for (int v = 0; v < VEC; ++v)
#pragma unroll
                    for (int c = 0; c < KC; ++c) acc[v][c] += uv[v] * tl[col * KC + c];
            }
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int64_t slot = sv + v;
            const int64_t dst = a.map ? a.map[slot] : slot;
            if (dst < 0) continue;
#pragma unroll
            for (int c = 0; c < KC; ++c)
                if (c < a.k) y[dst * a.ldy + c] = acc[v][c];
        }
    }
}

// ----------------------------------------------------------------- launchers
int64_t expand_smem_values(const MatvecArgs& a, int KC) {
    const int64_t TE = a.tile_e;
    int64_t vals = (TE > a.G ? TE : a.G) * KC;
    for (int l = 1; l <= a.nf; ++l) {
        const int64_t nodes_t = TE >= a.lv[l].n ? TE / a.lv[l].n : 1;
        vals += nodes_t * (int64_t)a.s * a.lv[l].r * KC;
    }
    return vals;
}

template <typename A, int KC, int PVEC, int EVEC>
cudaError_t run_kernel(int which, const MatvecArgs& a, cudaStream_t st) {
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(project_kernel<A, KC, PVEC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        cudaFuncSetAttribute(expand_kernel<A, KC, EVEC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr_done = true;
    }
    if (which == 0) {
        if (a.nf == 0) return cudaSuccess;
        const size_t psmem = (size_t)a.tile_p * KC * sizeof(A);
        const unsigned grid = (unsigned)(a.Np / a.tile_p);
        project_kernel<A, KC, PVEC><<<grid, 256, psmem, st>>>(a);
        return cudaGetLastError();
    }
    const size_t esmem = (size_t)expand_smem_values(a, KC) * sizeof(A);
    const unsigned egrid = (unsigned)(a.Np / a.tile_e);
    const int64_t want = a.tile_e / EVEC;
    const unsigned eblock = (unsigned)(want < 256 ? want : 256);
    expand_kernel<A, KC, EVEC><<<egrid, eblock, esmem, st>>>(a);
    return cudaGetLastError();
}

constexpr size_t kSmemCap = 227 * 1024;

template <typename A>
bool fits(const MatvecArgs& a, int KC) {
    return (size_t)a.tile_p * KC * sizeof(A) <= kSmemCap &&
           (size_t)expand_smem_values(a, KC) * sizeof(A) <= kSmemCap;
}

}  // namespace

int max_pass_rhs(int store_kind) { return store_kind == ST_F64 ? 32 : 64; }

// Launches kernel `which` (0 = project, 1 = expand) with the compiled RHS
// width a.kc (the pass width chosen by pass_width); a.k <= a.kc.
int launch_kernel(int which, int store_kind, const MatvecArgs& a, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (store_kind == ST_F64) {
        switch (a.kc) {
            case 1: return run_kernel<double, 1, 2, 2>(which, a, st);
            case 2: return run_kernel<double, 2, 2, 2>(which, a, st);
            case 4: return run_kernel<double, 4, 2, 1>(which, a, st);
            case 8: return run_kernel<double, 8, 2, 1>(which, a, st);
            case 16: return run_kernel<double, 16, 2, 1>(which, a, st);
            case 32: return run_kernel<double, 32, 2, 1>(which, a, st);
        }
        return (int)cudaErrorInvalidValue;
    }
    if (store_kind == ST_F32) {
        switch (a.kc) {
            case 1: return run_kernel<float, 1, 4, 4>(which, a, st);
            case 2: return run_kernel<float, 2, 4, 4>(which, a, st);
            case 4: return run_kernel<float, 4, 4, 2>(which, a, st);
            case 8: return run_kernel<float, 8, 4, 1>(which, a, st);
            case 16: return run_kernel<float, 16, 4, 1>(which, a, st);
            case 32: return run_kernel<float, 32, 4, 1>(which, a, st);
            case 64: return run_kernel<float, 64, 4, 1>(which, a, st);
        }
        return (int)cudaErrorInvalidValue;
    }
    return (int)cudaErrorNotSupported;
}

// Widest RHS pass the kernels can stage in shared memory for this geometry.
int pass_width(int store_kind, const MatvecArgs& a, int k) {
    static const int widths[] = {1, 2, 4, 8, 16, 32, 64};
    int best = 0;
    for (int w : widths) {
        if (w > max_pass_rhs(store_kind)) break;
        if (!(store_kind == ST_F64 ? fits<double>(a, w) : fits<float>(a, w))) break;
        best = w;
        if (w >= k) break;
    }
    return best;
}

// ------------------------------------------------------- static scratch
// Partial-sum scratch of hmat_matvec_noalloc: a fixed array in the
// library's device image, present on every GPU that loads the library until
// the process exits.  In host code `g_static_scratch` only names the symbol;
// its device address comes from cudaGetSymbolAddress, taken once per device
// (with that device current) and cached.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

int static_scratch_address(int device, void** ptr) {
    static std::mutex mu;
    static void* cached[128] = {};
    if (device < 0 || device >= 128) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!cached[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return (int)e;
        cached[device] = p;
    }
    *ptr = cached[device];
    return 0;
}

}  // namespace hm

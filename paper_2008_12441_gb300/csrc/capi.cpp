// The C ABI (include/hmat.h): argument checks, build orchestration, device
// upload, pass splitting, workspace clones with the cross-stream check,
// batched plans, save / load and introspection.  Every step of a product
// runs in the CUDA kernels (stream.cu, tc_matvec.cu, matvec.cu, gemv.cu);
// there is no host fallback.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>

#include "hm_device.h"
#include "hm_internal.h"
#include "philox_hm.h"

namespace hm {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int default_threads() {
    const unsigned n = std::thread::hardware_concurrency();
    return n ? (int)n : 4;
}

void parallel_for(int64_t n, int threads, const std::function<void(int64_t)>& fn) {
    if (n <= 0) return;
    int nt = threads > 0 ? threads : default_threads();
    if ((int64_t)nt > n) nt = (int)n;
    if (nt <= 1) {
        for (int64_t i = 0; i < n; ++i) fn(i);
        return;
    }
    std::atomic<int64_t> next{0};
    std::vector<std::thread> pool;
    pool.reserve(nt);
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&]() {
            for (;;) {
                const int64_t i = next.fetch_add(1);
                if (i >= n) break;
                fn(i);
            }
        });
    for (auto& th : pool) th.join();
}

namespace {
std::atomic<int64_t> g_launches{0};
// allocation-failure injection (hmat_inject_alloc_failure): allocations
// left before the failing one, negative when off
std::atomic<int64_t> g_fail_after{-1};
}
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

bool injected_alloc_failure() {
    int64_t v = g_fail_after.load(std::memory_order_relaxed);
    while (v >= 0) {
        if (g_fail_after.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 0;
    }
    return false;
}

}  // namespace hm

using namespace hm;

struct hmat_s {
    hmat_opts opts{};
    int kernel = 0, rank = 0, leaf_size = 0;
    double tol = 0.0;
    Tree tree;
    Geometry geo;
    Master master;
    bool have_master = false;
    bool device_fill = false;        // random fill generated on the device (no master arrays)
    int store = ST_F32;
    bool on_device = false;
    // device buffers
    void* dU = nullptr;
    void* dV = nullptr;
    void* dD = nullptr;
    void* dU_lo = nullptr;           // split bf16: low parts
    void* dV_lo = nullptr;
    void* dD_lo = nullptr;
    float* dscU = nullptr;           // bf16: per block; e4m3: per column
    float* dscV = nullptr;
    float* dscD = nullptr;           // per near-field group (bf16 dense blocks)
    std::vector<int64_t> sc_off;     // per level offset into the scale arrays
    int* d_stencil = nullptr;        // standard admissibility: interaction-list table (device)
    int64_t* d_map_orig = nullptr;   // slot -> original index or -1
    int64_t* d_map_tree = nullptr;   // slot -> tree position or -1
    void* dT = nullptr;
    int* dcnt = nullptr;             // arrival counters of the project kernel
    int* dstatus = nullptr;          // status word of the tensor-core kernels
    void* dxprep = nullptr;          // tensor-core path: prepared bf16 x tiles (and low parts)
    void* dxprep_lo = nullptr;
    void* dttprep = nullptr;         // prepared bf16 summed t per target node
    void* dttprep_lo = nullptr;
    std::vector<int64_t> tt_off;     // per level offset into dttprep (elements)
    void* dtmaps = nullptr;          // tensor maps of V, U, D for the streamed kernels
    std::vector<int> tma_rb;         // per level rows of one V box (empty: no project maps)
    std::vector<int> tma_rb_u;       // per level rows of one U box (empty: no expand maps)
    int tma_rb_d = 0;                // rows of one D box
    bool tc_maps = false;            // swizzled V maps of the tensor-core project
    bool fp8_maps = false;           // e4m3 V maps of the tensor-core project
    void* dX = nullptr;              // host-entry staging, N x max_nrhs
    void* dY = nullptr;
    int* hstatus = nullptr;          // pinned host copy of the status word (host entry point)
    // transposed product (HMAT_TRANSPOSE): the near-field blocks transposed
    // (null when every one is symmetric: D serves both products) and the
    // tensor maps over the swapped factor arrays; prepared once, on the
    // handle that owns the factors
    bool dense_sym = false;
    void* dDT = nullptr;
    void* dDT_lo = nullptr;
    void* dtmaps_t = nullptr;
    bool t_ready = false;
    std::mutex t_mu;
    unsigned last_path = 0;          // kernel families of the last product (hmat_last_path)
    int64_t device_bytes = 0, workspace_bytes = 0;
    int64_t tile_e = 0;
    // per-kernel timing (hmat_profile): event pairs around each launch
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[2];
    int64_t prof_launches[2] = {0, 0};
    double prof_ms[2] = {0.0, 0.0};
    // workspace clones (hmat_clone_workspace): a clone borrows the device
    // factors, scales, slot maps and tensor maps of `base` and owns only its
    // workspace (partial sums, counters, status word, prepared operands,
    // staging)
    hmat_s* base = nullptr;
    std::atomic<int> clones{0};      // live clones borrowing this handle's factors
    // the last product's stream and an event recorded after it: a product on
    // another stream while that event is pending would share the workspace
    cudaEvent_t busy_ev = nullptr;
    cudaStream_t busy_st = nullptr;
    bool busy_set = false;
};

namespace {

#define CU_TRY(call)                                                              \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            set_error("%s failed: %s", #call, cudaGetErrorString(e_));            \
            return HMAT_ECUDA;                                                    \
        }                                                                         \
    } while (0)

int dev_alloc(void** p, size_t bytes, int64_t& acc) {
    if (bytes == 0) bytes = 256;
    if (injected_alloc_failure()) {
        *p = nullptr;
        set_error("cudaMalloc(%zu) failed: allocation failure injected for a test", bytes);
        return HMAT_ENOMEM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? HMAT_ENOMEM : HMAT_ECUDA;
    }
    acc += (int64_t)bytes;
    return HMAT_OK;
}

// The per-handle workspace: what a product writes besides y.
void free_workspace(hmat_s* h) {
    void* ptrs[] = {h->dT,     h->dcnt,      h->dX,      h->dY,        h->dstatus,
                    h->dxprep, h->dxprep_lo, h->dttprep, h->dttprep_lo};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->hstatus) cudaFreeHost(h->hstatus);
    h->hstatus = nullptr;
    h->dT = h->dX = h->dY = nullptr;
    h->dcnt = h->dstatus = nullptr;
    h->dxprep = h->dxprep_lo = h->dttprep = h->dttprep_lo = nullptr;
}

void free_device(hmat_s* h) {
    free_workspace(h);
    // a clone's factor buffers belong to its base
    void* ptrs[] = {h->dU,   h->dV,   h->dD,   h->dU_lo,      h->dV_lo,      h->dD_lo,
                    h->dscU, h->dscV, h->dscD, h->d_map_orig, h->d_map_tree, h->dtmaps,
                    h->dDT,  h->dDT_lo, h->dtmaps_t, h->d_stencil};
    if (!h->base)
        for (void* p : ptrs)
            if (p) cudaFree(p);
    h->dU = h->dV = h->dD = h->dU_lo = h->dV_lo = h->dD_lo = h->dT = h->dX = h->dY = nullptr;
    h->dscU = h->dscV = h->dscD = nullptr;
    h->d_map_orig = h->d_map_tree = nullptr;
    h->dcnt = nullptr;
    h->dstatus = nullptr;
    h->dxprep = h->dxprep_lo = h->dttprep = h->dttprep_lo = nullptr;
    h->dtmaps = nullptr;
    h->dDT = h->dDT_lo = h->dtmaps_t = nullptr;
    h->d_stencil = nullptr;
    h->t_ready = false;
    h->tma_rb.clear();
    h->tma_rb_u.clear();
}

// Geometries the tensor-core kernels accept (see tc_eligible): whole project
// tiles per node and per near-field group, 128-slot tiles.
bool tc_geometry(const hmat_s* h) {
    const Geometry& g = h->geo;
    if (h->store != ST_BF16 && h->store != ST_BF16X2 && h->store != ST_FP8) return false;
    if (g.adm != 0) return false;      // standard admissibility: streamed kernels only
    if (g.nf < 1 || g.G % 128 != 0 || g.Np % 128 != 0 || g.tile_p % 64 != 0) return false;
    if (g.G % g.tile_p != 0) return false;
    for (int l = 1; l <= g.nf; ++l)
        if (g.lv[l].n < g.tile_p) return false;
    return true;
}

int store_of_prec(int prec) {
    switch (prec) {
        case HMAT_FP64: return ST_F64;
        case HMAT_FP32: return ST_F32;
        case HMAT_BF16: return ST_BF16;
        case HMAT_BF16X2: return ST_BF16X2;
        case HMAT_FP8E4M3: return ST_FP8;
    }
    return -1;
}

size_t vec_elem_bytes(const hmat_s* h) { return h->store == ST_F64 ? 8 : 4; }

int upload_bytes(const void* src, size_t bytes, void** dst, int64_t& acc) {
    int rc = dev_alloc(dst, bytes, acc);
    if (rc) return rc;
    CU_TRY(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return HMAT_OK;
}

template <typename T>
int upload_converted(const std::vector<double>& src, void** dst, int64_t& acc) {
    std::vector<T> tmp(src.size());
    for (size_t i = 0; i < src.size(); ++i) tmp[i] = (T)src[i];
    return upload_bytes(tmp.data(), tmp.size() * sizeof(T), dst, acc);
}

double pow2_ceil(double m) {
    if (!(m > 0.0)) return 1.0;
    return std::ldexp(1.0, (int)std::ceil(std::log2(m)));
}

// Factor array of every level in the requested storage.  bf16: one power-of-
// two scale per block (node j, sibling slot q: r_l columns); e4m3: one float
// scale per column (max |entry| / 448).  Scales are laid out per level.
int upload_factor(hmat_s* h, const std::vector<double>& M, void** dst, void** dst_lo,
                  float** dsc, int64_t& acc) {
    const Geometry& g = h->geo;
    const size_t n = M.size();
    if (h->store == ST_F64) return upload_converted<double>(M, dst, acc);
    if (h->store == ST_F32) return upload_converted<float>(M, dst, acc);
    if (h->store == ST_BF16X2) {
        std::vector<uint16_t> hi(n), lo(n);
        to_bf16_split(M.data(), hi.data(), lo.data(), n);
        int rc = upload_bytes(hi.data(), n * 2, dst, acc);
        if (rc) return rc;
        return upload_bytes(lo.data(), n * 2, dst_lo, acc);
    }
    // per-level scales
    std::vector<float> sc;
    h->sc_off.assign(g.nf + 1, 0);
    std::vector<uint16_t> q16;
    std::vector<uint8_t> q8;
    if (h->store == ST_BF16) q16.resize(n);
    else q8.resize(n);
    for (int l = 1; l <= g.nf; ++l) {
        const LevelGeom& lg = g.lv[l];
        const int64_t sr = (int64_t)g.s * lg.r;
        h->sc_off[l] = (int64_t)sc.size();
        const int64_t groups_per_node = h->store == ST_BF16 ? g.s : sr;
        const int64_t cols_per_group = h->store == ST_BF16 ? lg.r : 1;
        sc.resize(sc.size() + lg.nodes * groups_per_node, 1.f);
        parallel_for(lg.nodes, h->opts.threads, [&](int64_t j) {
            for (int64_t q = 0; q < groups_per_node; ++q) {
                const int64_t off = lg.fac_off + (j * sr + q * cols_per_group) * lg.n;
                const int64_t len = cols_per_group * lg.n;
                double mx = 0.0;
                for (int64_t e = 0; e < len; ++e) mx = std::max(mx, std::fabs(M[off + e]));
                double scale;
                if (h->store == ST_BF16) {
                    scale = pow2_ceil(mx);
                    to_bf16(M.data() + off, q16.data() + off, (size_t)len, 1.0 / scale);
                } else {
                    scale = mx > 0.0 ? (double)(float)(mx / 448.0) : 1.0;
                    to_fp8e4m3(M.data() + off, q8.data() + off, (size_t)len, 1.0 / scale);
                }
                sc[h->sc_off[l] + j * groups_per_node + q] = (float)scale;
            }
        });
    }
    int rc = h->store == ST_BF16 ? upload_bytes(q16.data(), n * 2, dst, acc)
                                 : upload_bytes(q8.data(), n, dst, acc);
    if (rc) return rc;
    return upload_bytes(sc.data(), std::max<size_t>(1, sc.size()) * sizeof(float),
                        reinterpret_cast<void**>(dsc), acc);
}

// Dense near-field blocks: float64/float32 as is; split bf16 as hi + lo;
// bf16 with one power-of-two scale per near-field group (over the blocks of
// all its source groups) in the bf16 and e4m3 modes.
int upload_dense(hmat_s* h, int64_t& acc) {
    const Geometry& g = h->geo;
    const std::vector<double>& D = h->master.D;
    const size_t n = D.size();
    // every near-field block symmetric (a symmetric kernel on the diagonal
    // groups): the transposed product reads D itself
    {
        std::atomic<bool> sym{true};
        const int64_t G = g.G, gg = G * G;
        if ((int64_t)n == g.groups * gg)
            parallel_for(g.groups, h->opts.threads, [&](int64_t gi) {
                const double* Dg = D.data() + gi * gg;
                for (int64_t b = 0; b < G && sym.load(std::memory_order_relaxed); ++b)
                    for (int64_t p = b + 1; p < G; ++p)
                        if (Dg[b * G + p] != Dg[p * G + b]) {
                            sym.store(false, std::memory_order_relaxed);
                            break;
                        }
            });
        h->dense_sym = (int64_t)n == g.groups * gg && sym.load();
    }
    if (h->store == ST_F64) return upload_converted<double>(D, &h->dD, acc);
    if (h->store == ST_F32) return upload_converted<float>(D, &h->dD, acc);
    if (h->store == ST_BF16X2) {
        std::vector<uint16_t> hi(n), lo(n);
        to_bf16_split(D.data(), hi.data(), lo.data(), n);
        int rc = upload_bytes(hi.data(), n * 2, &h->dD, acc);
        if (rc) return rc;
        return upload_bytes(lo.data(), n * 2, &h->dD_lo, acc);
    }
    std::vector<uint16_t> q16(n);
    // one scale per target group over all its source groups' blocks
    std::vector<float> sc(g.groups, 1.f);
    const int64_t gg = g.nnb * g.G * g.G;
    parallel_for(g.groups, h->opts.threads, [&](int64_t gi) {
        double mx = 0.0;
        for (int64_t e = 0; e < gg; ++e) mx = std::max(mx, std::fabs(D[gi * gg + e]));
        const double scale = pow2_ceil(mx);
        to_bf16(D.data() + gi * gg, q16.data() + gi * gg, (size_t)gg, 1.0 / scale);
        sc[gi] = (float)scale;
    });
    int rc = upload_bytes(q16.data(), n * 2, &h->dD, acc);
    if (rc) return rc;
    return upload_bytes(sc.data(), sc.size() * sizeof(float), reinterpret_cast<void**>(&h->dscD),
                        acc);
}

// bytes of one stored factor element
int factor_elem_bytes(int store) {
    switch (store) {
        case ST_F64: return 8;
        case ST_F32: return 4;
        case ST_FP8: return 1;
        default: return 2;
    }
}

// Factor arrays a set of tensor maps describes, and the encoded set.
struct MapPtrs {
    const void *U, *V, *D, *U_lo, *V_lo, *D_lo;
};
struct MapSet {
    std::vector<unsigned char> maps;
    std::vector<int> rb, rbu;
    int rbd = 0;
    bool proj = false, expd = false, tc = false, fp8 = false;
};

// Encodes every tensor map of the factor arrays `p` (the handle's own, or
// U and V swapped with the transposed dense blocks for K^T) into `m`.
void encode_maps(const hmat_s* h, const MapPtrs& p, MapSet& m) {
    const Geometry& g = h->geo;
    if (g.nf < 1) return;
    const int es = factor_elem_bytes(h->store);
    const int esd = h->store == ST_FP8 ? 2 : es;          // dense blocks: bf16 in the e4m3 mode
    const int parts = h->store == ST_BF16X2 ? 2 : 1;
    std::vector<unsigned char> maps((size_t)kTensorMapKinds * (kMaxLevels + 1) * kTensorMapBytes, 0);
    auto map_at = [&](int kind, int l) {
        return maps.data() + ((size_t)kind * (kMaxLevels + 1) + l) * kTensorMapBytes;
    };
    bool proj = true, expd = g.G % kExpandStreamTile == 0;
    for (int l = 1; l <= g.nf; ++l) {
        if (g.lv[l].r > 0 && g.lv[l].n < g.tile_p) proj = false;
        if (g.lv[l].r > 0 && g.lv[l].n < kExpandStreamTile) expd = false;
    }
    std::vector<int> rb(g.nf + 1, 0), rbu(g.nf + 1, 0);
    int rbd = 0;
    const int cap = stream_stage_rows(g.tile_p, es, parts);
    for (int l = 1; l <= g.nf && (proj || expd); ++l) {
        const LevelGeom& lg = g.lv[l];
        if (lg.r == 0) continue;
        const int sr = g.s * lg.r;
        rb[l] = stream_box_rows(sr, cap);
        rbu[l] = expand_box_rows(sr, es, parts);
        for (int part = 0; part < parts; ++part) {
            const char* vb = static_cast<const char*>(part ? p.V_lo : p.V) + lg.fac_off * es;
            const char* ub = static_cast<const char*>(part ? p.U_lo : p.U) + lg.fac_off * es;
            if (proj && encode_rows_map(map_at(part, l), vb, es, (uint64_t)lg.n, (uint64_t)(lg.nodes * sr),
                                        (uint32_t)g.tile_p, (uint32_t)rb[l], false))
                proj = false;
            if (expd && encode_rows_map(map_at(2 + part, l), ub, es, (uint64_t)lg.n, (uint64_t)(lg.nodes * sr),
                                        (uint32_t)kExpandStreamTile, (uint32_t)rbu[l], false))
                expd = false;
        }
    }
    if (expd) {
        // rows of the dense blocks: group g, source column c < nnb G at g nnb G + c
        rbd = expand_box_rows((int)(g.nnb * g.G), esd, parts);
        for (int part = 0; part < parts && expd; ++part) {
            const void* db = part ? p.D_lo : p.D;
            if (encode_rows_map(map_at(2 + part, 0), db, esd, (uint64_t)g.G, (uint64_t)(g.groups * g.nnb * g.G),
                                (uint32_t)kExpandStreamTile, (uint32_t)rbd, false))
                expd = false;
        }
    }
    // e4m3 V maps of the tensor-core project (widened to bf16 in shared memory)
    if (h->store == ST_FP8 && tc_geometry(h)) {
        bool ok8 = true;
        for (int l = 1; l <= g.nf && ok8; ++l) {
            const LevelGeom& lg = g.lv[l];
            if (lg.r == 0) continue;
            const int sr = g.s * lg.r;
            const char* vb = static_cast<const char*>(p.V) + lg.fac_off;
            if (encode_rows_map(map_at(kMapV8, l), vb, 1, (uint64_t)lg.n, (uint64_t)(lg.nodes * sr), 64, 128,
                                false))
                ok8 = false;
            if (ok8 && sr % 128 != 0 &&
                encode_rows_map(map_at(kMapV8Rem, l), vb, 1, (uint64_t)lg.n, (uint64_t)(lg.nodes * sr), 64,
                                (uint32_t)(sr % 128), false))
                ok8 = false;
            // U for the expand: raw e4m3 boxes of 64 slots x 64 columns
            const char* ub = static_cast<const char*>(p.U) + lg.fac_off;
            const int rem = (sr % 64 + 15) / 16 * 16;
            if (ok8 && encode_rows_map(map_at(kMapU8, l), ub, 1, (uint64_t)lg.n, (uint64_t)(lg.nodes * sr), 64, 64,
                                       false))
                ok8 = false;
            if (ok8 && rem != 0 &&
                encode_rows_map(map_at(kMapU8Rem, l), ub, 1, (uint64_t)lg.n, (uint64_t)(lg.nodes * sr), 64,
                                (uint32_t)rem, false))
                ok8 = false;
        }
        // the near-field blocks stay bf16: swizzled map as for bf16 storage
        if (ok8 && encode_rows_map(map_at(kMapUSw, 0), p.D, 2, (uint64_t)g.G, (uint64_t)(g.groups * g.G), 64, 64,
                                   true))
            ok8 = false;
        m.fp8 = ok8;
    }
    // swizzled V maps of the tensor-core project (bf16 storage)
    bool tcm = (h->store == ST_BF16 || h->store == ST_BF16X2) && tc_geometry(h);
    for (int l = 1; l <= g.nf && tcm; ++l) {
        const LevelGeom& lg = g.lv[l];
        if (lg.r == 0) continue;
        const int sr = g.s * lg.r;
        for (int part = 0; part < parts && tcm; ++part) {
            const char* vb = static_cast<const char*>(part ? p.V_lo : p.V) + lg.fac_off * es;
            if (encode_rows_map(map_at(kMapVSw + part, l), vb, es, (uint64_t)lg.n, (uint64_t)(lg.nodes * sr), 64,
                                128, true))
                tcm = false;
            if (tcm && sr % 128 != 0 &&
                encode_rows_map(map_at(kMapVSwRem + part, l), vb, es, (uint64_t)lg.n, (uint64_t)(lg.nodes * sr),
                                64, (uint32_t)(sr % 128), true))
                tcm = false;
        }
    }
    // swizzled U and D maps of the tensor-core expand
    const int kb = tc_expand_kb(h->store);
    for (int l = 0; l <= g.nf && tcm; ++l) {
        const int cols = l == 0 ? (int)g.G : g.s * g.lv[l].r;
        if (l > 0 && g.lv[l].r == 0) continue;
        const int64_t rows = l == 0 ? g.groups * g.G : g.lv[l].nodes * cols;
        const uint64_t len = l == 0 ? (uint64_t)g.G : (uint64_t)g.lv[l].n;
        const int rem = (cols % kb + 15) / 16 * 16;
        for (int part = 0; part < parts && tcm; ++part) {
            const void* base = l == 0 ? (part ? p.D_lo : p.D)
                                      : static_cast<const void*>(static_cast<const char*>(part ? p.U_lo : p.U) +
                                                                 g.lv[l].fac_off * es);
            if (encode_rows_map(map_at(kMapUSw + part, l), base, es, len, (uint64_t)rows, 64, (uint32_t)kb, true))
                tcm = false;
            if (tcm && rem != 0 &&
                encode_rows_map(map_at(kMapUSwRem + part, l), base, es, len, (uint64_t)rows, 64, (uint32_t)rem, true))
                tcm = false;
        }
    }
    m.tc = tcm || m.fp8;
    m.proj = proj;
    m.expd = expd;
    m.rb = rb;
    m.rbu = rbu;
    m.rbd = rbd;
    m.maps = std::move(maps);
}

// Tensor maps for the streamed single-right-hand-side kernels: over the
// rows of every level of V (project; when every level's nodes span whole
// project tiles) and of U and the dense blocks (expand; when the
// near-field group is a multiple of the expand tile), and the swizzled
// maps of the tensor-core kernels.  A geometry without them, or a driver
// that does not encode them, keeps the cached kernels.
int upload_tensor_maps(hmat_s* h, int64_t& ws) {
    h->tma_rb.clear();
    h->tma_rb_u.clear();
    h->tma_rb_d = 0;
    h->tc_maps = false;
    h->fp8_maps = false;
    MapSet m;
    encode_maps(h, MapPtrs{h->dU, h->dV, h->dD, h->dU_lo, h->dV_lo, h->dD_lo}, m);
    h->fp8_maps = m.fp8;
    h->tc_maps = m.tc;
    if (!m.proj && !m.expd && !m.tc) return HMAT_OK;
    int rc = dev_alloc(&h->dtmaps, m.maps.size(), ws);
    if (rc) return rc;
    CU_TRY(cudaMemcpy(h->dtmaps, m.maps.data(), m.maps.size(), cudaMemcpyHostToDevice));
    if (m.proj) h->tma_rb = m.rb;
    if (m.expd) {
        h->tma_rb_u = m.rbu;
        h->tma_rb_d = m.rbd;
    }
    return HMAT_OK;
}

// The transposed product's device state on the handle `b` that owns the
// factors: under weak admissibility block (j, i) of K^T is V_ij U_ij^T and
// the slot of i at j has the formula of the slot of j at i, so K^T uses the
// same kernels with the U and V arrays (and their scales) swapped; the
// near-field groups need D_g^T, a device-side transposed copy unless every
// group is symmetric.  Allocates, and synchronises the device.
int prepare_transpose(hmat_s* b) {
    std::lock_guard<std::mutex> lock(b->t_mu);
    if (b->t_ready) return HMAT_OK;
    if (b->geo.adm) {
        set_error("the transposed product is built for weak admissibility only");
        return HMAT_EUNSUPPORTED;
    }
    CU_TRY(cudaSetDevice(b->opts.device));
    const Geometry& g = b->geo;
    int64_t acc = 0;
    int rc;
    if (!b->dense_sym && g.groups > 0) {
        const int esd = b->store == ST_FP8 ? 2 : factor_elem_bytes(b->store);
        const size_t bytes = (size_t)g.groups * g.G * g.G * esd;
        if ((rc = dev_alloc(&b->dDT, bytes, acc))) return rc;
        int e = transpose_groups(b->dD, b->dDT, esd, g.groups, g.G, nullptr);
        if (e == 0 && b->dD_lo) {
            if ((rc = dev_alloc(&b->dDT_lo, bytes, acc))) return rc;
            e = transpose_groups(b->dD_lo, b->dDT_lo, esd, g.groups, g.G, nullptr);
        }
        if (e != 0) {
            set_error("transpose of the near-field blocks failed: %s", cudaGetErrorString((cudaError_t)e));
            return HMAT_ECUDA;
        }
        CU_TRY(cudaDeviceSynchronize());
    }
    const void* Dt = b->dDT ? b->dDT : b->dD;
    const void* Dt_lo = b->dDT_lo ? b->dDT_lo : b->dD_lo;
    MapSet m;
    encode_maps(b, MapPtrs{b->dV, b->dU, Dt, b->dV_lo, b->dU_lo, Dt_lo}, m);
    // the swapped arrays have the same shapes: the same boxes and kernels
    const bool same = m.proj == !b->tma_rb.empty() && m.expd == !b->tma_rb_u.empty() && m.tc == b->tc_maps &&
                      (!m.proj || m.rb == b->tma_rb) && (!m.expd || (m.rbu == b->tma_rb_u && m.rbd == b->tma_rb_d));
    if (!same) {
        set_error("tensor maps of the transposed arrays differ from the handle's");
        return HMAT_ECUDA;
    }
    if (!b->dtmaps) {
        b->device_bytes += acc;
        b->t_ready = true;
        return HMAT_OK;
    }
    if ((rc = dev_alloc(&b->dtmaps_t, m.maps.size(), acc))) return rc;
    CU_TRY(cudaMemcpy(b->dtmaps_t, m.maps.data(), m.maps.size(), cudaMemcpyHostToDevice));
    b->device_bytes += acc;
    b->t_ready = true;
    return HMAT_OK;
}

// Right-hand sides the partial-sum buffer holds per pass: the pass widths
// are powers of two (the compiled widths of the CUDA-core kernels, and the
// tensor-core kernels' rounding), so max_nrhs rounded up to one.
int workspace_width(const hmat_s* h) {
    const int k = std::min(h->opts.max_nrhs, max_pass_rhs(h->store));
    int w = 1;
    while (w < k) w *= 2;
    return w;
}

// Allocates the workspace of a handle whose geometry (and, for the
// tensor-core geometries, tt_off) is set: partial sums and arrival
// counters for max_nrhs right-hand sides, the status word, the prepared
// tensor-core operands and the host-entry staging of x and y.
int alloc_workspace(hmat_s* h, int64_t& ws) {
    const Geometry& g = h->geo;
    int rc;
    const size_t acc_bytes = h->store == ST_F64 ? 8 : 4;
    const int kc = workspace_width(h);
    if ((rc = dev_alloc(&h->dT, (size_t)std::max<int64_t>(1, g.t_per_rhs) * kc * acc_bytes, ws)))
        return rc;
    if ((rc = dev_alloc((void**)&h->dcnt, (size_t)std::max<int64_t>(1, g.counters) * sizeof(int), ws)))
        return rc;
    CU_TRY(cudaMemset(h->dcnt, 0, (size_t)std::max<int64_t>(1, g.counters) * sizeof(int)));
    if ((rc = dev_alloc((void**)&h->dstatus, sizeof(int), ws))) return rc;
    CU_TRY(cudaMemset(h->dstatus, 0, sizeof(int)));
    if (tc_geometry(h)) {
        // prepared bf16 B operands of the tensor-core kernels (64 right-hand sides)
        const bool split = h->store == ST_BF16X2;
        const size_t xb = (size_t)g.Np * 64 * 2;
        int64_t tt = 0;
        for (int l = 1; l <= g.nf; ++l) {
            const int64_t srp = ((int64_t)g.s * g.lv[l].r + 63) / 64 * 64;
            tt += g.lv[l].nodes * 64 * srp;
        }
        const size_t tb = (size_t)std::max<int64_t>(1, tt) * 2;
        if ((rc = dev_alloc(&h->dxprep, xb, ws))) return rc;
        // the padding columns of every region must read as zero: written once here
        if ((rc = dev_alloc(&h->dttprep, tb, ws))) return rc;
        CU_TRY(cudaMemset(h->dttprep, 0, tb));
        if (split) {
            if ((rc = dev_alloc(&h->dxprep_lo, xb, ws))) return rc;
            if ((rc = dev_alloc(&h->dttprep_lo, tb, ws))) return rc;
            CU_TRY(cudaMemset(h->dttprep_lo, 0, tb));
        }
    }
    const size_t vb = (size_t)h->tree.N * h->opts.max_nrhs * vec_elem_bytes(h);
    if ((rc = dev_alloc(&h->dX, vb, ws))) return rc;
    if ((rc = dev_alloc(&h->dY, vb, ws))) return rc;
    if (injected_alloc_failure() ||
        cudaHostAlloc((void**)&h->hstatus, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        h->hstatus = nullptr;
        set_error("cudaHostAlloc of the status word failed");
        return HMAT_ENOMEM;
    }
    *h->hstatus = 0;
    return HMAT_OK;
}

// The random fill written straight into the device layout (FP32 / FP64
// storage, unpadded tree, weak admissibility): bit-identical to the host
// fill, without its float64 master.
int fill_on_device(hmat_s* h) {
    const Geometry& g = h->geo;
    const bool f64 = h->store == ST_F64;
    const size_t es = f64 ? 8 : 4;
    int rc;
    if ((rc = dev_alloc(&h->dU, (size_t)std::max<int64_t>(1, g.fac_entries) * es, h->device_bytes))) return rc;
    if ((rc = dev_alloc(&h->dV, (size_t)std::max<int64_t>(1, g.fac_entries) * es, h->device_bytes))) return rc;
    if ((rc = dev_alloc(&h->dD, (size_t)std::max<int64_t>(1, g.dense_entries) * es, h->device_bytes))) return rc;
    const int nc = 1 << g.d;
    const uint64_t seed = h->opts.seed;
    for (int l = 1; l <= g.nf; ++l) {
        const LevelGeom& lg = g.lv[l];
        if (lg.r == 0) continue;
        const size_t off = (size_t)lg.fac_off * es;
        int e = fill_random_factor(static_cast<char*>(h->dU) + off, f64, RAND_U, seed, l, lg.nodes, lg.n, g.s,
                                   lg.r, rand_scale(lg.r));
        if (e == 0)
            e = fill_random_factor(static_cast<char*>(h->dV) + off, f64, RAND_V, seed, l, lg.nodes, lg.n, g.s, lg.r,
                                   rand_scale(lg.n));
        if (e != 0) { set_error("hmat_build: device fill failed: %s", cudaGetErrorString((cudaError_t)e)); return HMAT_ECUDA; }
    }
    const bool leaf_pairs = !h->opts.leaf_lowrank;
    const int e = fill_random_dense(h->dD, f64, seed, leaf_pairs ? g.L : g.nf, g.groups, g.G, g.m_pad, nc,
                                    leaf_pairs ? 1 : 0, rand_scale(leaf_pairs ? g.m_pad : g.G));
    if (e != 0) { set_error("hmat_build: device fill failed: %s", cudaGetErrorString((cudaError_t)e)); return HMAT_ECUDA; }
    CU_TRY(cudaDeviceSynchronize());
    h->dense_sym = false;
    return HMAT_OK;
}

int upload(hmat_s* h) {
    CU_TRY(cudaSetDevice(h->opts.device));
    const Geometry& g = h->geo;
    int rc;
    if (h->device_fill) {
        if ((rc = fill_on_device(h))) return rc;
    } else {
        if ((rc = upload_factor(h, h->master.U, &h->dU, &h->dU_lo, &h->dscU, h->device_bytes))) return rc;
        if ((rc = upload_factor(h, h->master.V, &h->dV, &h->dV_lo, &h->dscV, h->device_bytes))) return rc;
        if ((rc = upload_dense(h, h->device_bytes))) return rc;
    }
    int64_t ws = 0;
    if ((rc = dev_alloc((void**)&h->d_map_orig, g.Np * sizeof(int64_t), ws))) return rc;
    if ((rc = dev_alloc((void**)&h->d_map_tree, g.Np * sizeof(int64_t), ws))) return rc;
    CU_TRY(cudaMemcpy(h->d_map_orig, h->tree.slot_src.data(), g.Np * sizeof(int64_t),
                      cudaMemcpyHostToDevice));
    std::vector<int64_t> mt(g.Np, -1);
    for (int64_t p = 0; p < h->tree.N; ++p) mt[h->tree.slot[p]] = p;
    CU_TRY(cudaMemcpy(h->d_map_tree, mt.data(), g.Np * sizeof(int64_t), cudaMemcpyHostToDevice));
    if ((rc = upload_tensor_maps(h, ws))) return rc;
    if (g.adm) {
        // standard admissibility runs on the streamed kernels only
        if (h->tma_rb.empty() || h->tma_rb_u.empty()) {
            set_error("hmat_build: standard admissibility needs the streamed kernels' geometry "
                      "(near-field groups and level nodes of whole 256-slot tiles)");
            return HMAT_EUNSUPPORTED;
        }
        Stencil st;
        build_stencil(g.d, st);
        if ((rc = upload_bytes(st.packed.data(), st.packed.size() * sizeof(int), (void**)&h->d_stencil, ws)))
            return rc;
    }
    if (tc_geometry(h)) {
        // offsets of the prepared summed t per level (64 rows x s r_l rounded up to 64)
        h->tt_off.assign(g.nf + 1, 0);
        int64_t tt = 0;
        for (int l = 1; l <= g.nf; ++l) {
            h->tt_off[l] = tt;
            const int64_t srp = ((int64_t)g.s * g.lv[l].r + 63) / 64 * 64;
            tt += g.lv[l].nodes * 64 * srp;
        }
    }
    if ((rc = alloc_workspace(h, ws))) return rc;
    h->workspace_bytes = ws;
    h->on_device = true;
    return HMAT_OK;
}

// Stream-conflict check of a product on `st`: refused while the handle's
// previous product, issued on another stream, has not completed (both
// would use the same workspace).  Skipped while `st` is being captured
// into a graph.
int claim_stream(hmat_s* h, cudaStream_t st, bool* capturing, const char* who) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusNone;
    }
    *capturing = cs != cudaStreamCaptureStatusNone;
    if (*capturing || !h->busy_set || h->busy_st == st) return HMAT_OK;
    const cudaError_t q = cudaEventQuery(h->busy_ev);
    if (q == cudaSuccess) return HMAT_OK;
    if (q == cudaErrorNotReady) {
        set_error("%s: the handle's previous product on another stream has not completed; "
                  "synchronize, or give each stream its own hmat_clone_workspace",
                  who);
        return HMAT_EUNSUPPORTED;
    }
    set_error("%s: cudaEventQuery: %s", who, cudaGetErrorString(q));
    return HMAT_ECUDA;
}

// Records the end of a product on `st` (see claim_stream).
void release_stream(hmat_s* h, cudaStream_t st, bool capturing) {
    if (capturing) return;
    if (!h->busy_ev && cudaEventCreateWithFlags(&h->busy_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        h->busy_ev = nullptr;
        return;
    }
    if (cudaEventRecord(h->busy_ev, st) == cudaSuccess) {
        h->busy_st = st;
        h->busy_set = true;
    } else {
        cudaGetLastError();
    }
}

// Kernel arguments of one product (everything but the pass-dependent x, y,
// k, kc and the partial-sum buffers).
void fill_args(const hmat_s* h, int flags, MatvecArgs& a) {
    const Geometry& g = h->geo;
    std::memset(&a, 0, sizeof(a));
    a.d = g.d;
    a.s = g.s;
    a.nf = g.nf;
    a.adm = g.adm;
    a.nnb = g.nnb;
    a.stencil = h->d_stencil;
    a.store = h->store;
    a.Np = g.Np;
    a.G = g.G;
    a.tile_p = g.tile_p;
    a.tile_e = g.tile_p;
    for (int l = 1; l <= g.nf; ++l) {
        const LevelGeom& lg = g.lv[l];
        a.lv[l].r = lg.r;
        a.lv[l].nsub = lg.nsub;
        a.lv[l].n = lg.n;
        a.lv[l].fac_off = lg.fac_off;
        a.lv[l].fin_off = lg.fin_off;
        a.lv[l].part_off = lg.part_off;
        a.lv[l].cnt_off = lg.cnt_off;
        a.lv[l].sc_off = l < (int)h->sc_off.size() ? h->sc_off[l] : 0;
        a.lv[l].tt_off = l < (int)h->tt_off.size() ? h->tt_off[l] : 0;
        a.lv[l].tma_rb = l < (int)h->tma_rb.size() ? h->tma_rb[l] : 0;
        a.lv[l].tma_rb_u = l < (int)h->tma_rb_u.size() ? h->tma_rb_u[l] : 0;
    }
    // K^T (prepared on the handle owning the factors): U and V swapped, the
    // transposed near-field blocks, the maps over those arrays
    const hmat_s* own = h->base ? h->base : h;
    const bool tr = (flags & HMAT_TRANSPOSE) != 0 && own->t_ready;
    const void* maps = tr ? own->dtmaps_t : h->dtmaps;
    a.tmaps = h->tma_rb.empty() ? nullptr : maps;
    a.tmaps_u = h->tma_rb_u.empty() ? nullptr : maps;
    a.tmaps_tc = h->tc_maps ? maps : nullptr;
    // per-kernel event timing (hmat_profile) puts events between the
    // kernels: launch them plainly then
    a.pdl = h->prof ? 0 : 1;
    a.tma_rb_d = h->tma_rb_d;
    a.xprep = h->dxprep;
    a.xprep_lo = h->dxprep_lo;
    a.ttprep = h->dttprep;
    a.ttprep_lo = h->dttprep_lo;
    a.U = tr ? h->dV : h->dU;
    a.V = tr ? h->dU : h->dV;
    a.D = tr && own->dDT ? own->dDT : h->dD;
    a.U_lo = tr ? h->dV_lo : h->dU_lo;
    a.V_lo = tr ? h->dU_lo : h->dV_lo;
    a.D_lo = tr && own->dDT_lo ? own->dDT_lo : h->dD_lo;
    a.scU = tr ? h->dscV : h->dscU;
    a.scV = tr ? h->dscU : h->dscV;
    a.scD = h->dscD;
    const bool tree_order = (flags & HMAT_TREE_ORDER) != 0;
    a.map = tree_order ? (g.Np == h->tree.N ? nullptr : h->d_map_tree) : h->d_map_orig;
    a.status = h->dstatus;
}

// Leaf slots: a multiple of the storage's alignment and of the caller's
// multiple q (both powers of two times small factors: their least common
// multiple).
int leaf_multiple(int store, int q) {
    const int a = slot_align(store);
    if (q <= 0) return a;
    int x = a, y = q;
    while (y) { const int t = x % y; x = y; y = t; }
    return a / x * q;
}

// Pass width: the tensor-core kernels take any k <= 64 in one pass.
int choose_pass(const MatvecArgs& a, int k) {
    if (k >= 2 && a.status && tc_eligible(a)) {
        int w = 2;
        while (w < k && w < 64) w *= 2;
        return w;
    }
    return pass_width(a, k);
}

// expand tile: m_pad * 2^a slots with 256 * VEC threads at most
int64_t choose_tile_e(const Geometry& g) {
    int64_t te = g.m_pad;
    while (te * 2 <= 1024 && te * 2 <= g.Np) te *= 2;
    return te;
}

}  // namespace

extern "C" {

void hmat_default_opts(hmat_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->prec = HMAT_FP32;
    o->method = HMAT_RSVD;
    o->leaf_lowrank = 0;
    o->oversample = 8;
    o->power_iters = 1;
    o->device = 0;
    o->max_nrhs = 64;
    o->threads = 0;
    o->keep_host = 0;
    o->build_gpu = -1;
    o->seed = 0;
    o->admissibility = HMAT_ADM_WEAK;
}

const char* hmat_last_error(void) { return g_err; }

int hmat_build(const double* points, int64_t N, int d, int kernel, int leaf_size, int rank,
               double tol, const hmat_opts* opts, hmat_t* out) {
    g_err[0] = 0;
    if (!points || !out) { set_error("hmat_build: null pointer"); return HMAT_EINVAL; }
    if (N < 1) { set_error("hmat_build: N must be >= 1"); return HMAT_EINVAL; }
    if (d != 2 && d != 3) { set_error("hmat_build: d must be 2 or 3"); return HMAT_EINVAL; }
    if (leaf_size < 1) { set_error("hmat_build: leaf_size must be >= 1"); return HMAT_EINVAL; }
    if (kernel == HMAT_K_LOG2D && d != 2) { set_error("hmat_build: log kernel needs d = 2"); return HMAT_EINVAL; }
    if (kernel == HMAT_K_INV4PIR_3D && d != 3) { set_error("hmat_build: 1/r kernel needs d = 3"); return HMAT_EINVAL; }
    if (kernel < 0 || kernel > 2) { set_error("hmat_build: unknown kernel"); return HMAT_EINVAL; }
    hmat_opts o;
    hmat_default_opts(&o);
    if (opts) o = *opts;
    if (store_of_prec(o.prec) < 0) { set_error("hmat_build: unknown precision"); return HMAT_EINVAL; }
    if (o.method < 0 || o.method > 2) { set_error("hmat_build: unknown method"); return HMAT_EINVAL; }
    if ((kernel == HMAT_K_RANDOM) != (o.method == HMAT_RANDOM_FILL)) {
        set_error("hmat_build: the random kernel goes with the random fill and only with it");
        return HMAT_EINVAL;
    }
    if (rank <= 0 && !(tol > 0.0)) { set_error("hmat_build: need rank > 0 or tol > 0"); return HMAT_EINVAL; }
    if (o.method == HMAT_RANDOM_FILL && rank <= 0) { set_error("hmat_build: random fill needs rank > 0"); return HMAT_EINVAL; }
    if (o.max_nrhs < 1 || o.oversample < 0 || o.power_iters < 0) { set_error("hmat_build: bad options"); return HMAT_EINVAL; }
    if (o.admissibility != HMAT_ADM_WEAK && o.admissibility != HMAT_ADM_STANDARD) {
        set_error("hmat_build: unknown admissibility condition");
        return HMAT_EINVAL;
    }
    if (o.leaf_slot_multiple < 0 || o.leaf_slot_multiple > 256 || o.leaf_slot_multiple % 8 != 0) {
        set_error("hmat_build: leaf_slot_multiple must be 0 or a multiple of 8 up to 256");
        return HMAT_EINVAL;
    }
    if (o.admissibility == HMAT_ADM_STANDARD && o.leaf_lowrank) {
        set_error("hmat_build: standard admissibility is built with dense leaf pairs (leaf_lowrank = 0)");
        return HMAT_EUNSUPPORTED;
    }
    for (int64_t i = 0; i < N * d; ++i)
        if (!std::isfinite(points[i])) { set_error("hmat_build: non-finite coordinate"); return HMAT_EINVAL; }
    if (tree_depth(N, d, leaf_size) > kMaxLevels - 1) { set_error("hmat_build: tree too deep"); return HMAT_EUNSUPPORTED; }
    std::unique_ptr<hmat_s> h;
    try {
        h.reset(new hmat_s());
        h->opts = o;
        h->kernel = kernel;
        h->rank = rank;
        h->tol = tol;
        h->leaf_size = leaf_size;
        h->store = store_of_prec(o.prec);
        build_tree(points, N, d, leaf_size, o.threads, leaf_multiple(h->store, o.leaf_slot_multiple), h->tree);
        std::vector<double> pts_tree((size_t)(N * d));
        for (int64_t p = 0; p < N; ++p)
            for (int k = 0; k < d; ++k) pts_tree[p * d + k] = points[h->tree.perm[p] * d + k];
        BuildParams bp;
        bp.kernel = kernel;
        bp.rank = rank;
        bp.tol = tol;
        bp.method = o.method;
        bp.oversample = o.oversample;
        bp.power_iters = o.power_iters;
        bp.leaf_lowrank = o.leaf_lowrank;
        bp.threads = o.threads;
        bp.seed = o.seed;
        bp.adm = o.admissibility;
        // the random fill written on the device: unpadded trees, weak
        // admissibility, FP32/FP64 storage, no host copy kept
        const bool fill_dev = o.device >= 0 && !o.keep_host && random_fill_on_device_ok(h->tree, bp) &&
                              (h->store == ST_F32 || h->store == ST_F64) &&
                              (o.build_gpu == 1 || (o.build_gpu < 0 && N >= 65536));
        if (fill_dev) {
            h->device_fill = true;
            random_fill_layout(h->tree, bp, h->geo, h->master);
            h->have_master = false;
            h->tile_e = choose_tile_e(h->geo);
            const int rc0 = upload(h.get());
            if (rc0) {
                free_device(h.get());
                return rc0;
            }
            *out = h.release();
            return HMAT_OK;
        }
        const bool want_gpu = o.device >= 0 && o.method == HMAT_RSVD &&
                              (o.build_gpu == 1 || (o.build_gpu < 0 && N >= 65536));
        GpuSketch* gs = nullptr;
        if (want_gpu) {
            std::vector<int64_t> orig(h->tree.perm);
            int rc0 = gpu_sketch_init(&gs, o.device, pts_tree.data(), orig.data(), N, d, kernel);
            if (rc0) {
                gpu_sketch_free(gs);
                return rc0;
            }
            bp.gpu = gs;
        }
        int rc = compress_all(h->tree, pts_tree.data(), bp, h->geo, h->master);
        gpu_sketch_free(gs);
        if (rc) return rc;
        h->have_master = true;
        h->tile_e = choose_tile_e(h->geo);
        if (o.device >= 0) {
            rc = upload(h.get());
            if (rc) {
                free_device(h.get());
                return rc;
            }
            if (!o.keep_host) {
                Master empty;
                empty.factor_entries = h->master.factor_entries;
                empty.dense_entries = h->master.dense_entries;
                empty.lowrank_blocks = h->master.lowrank_blocks;
                empty.dense_blocks = h->master.dense_blocks;
                h->master = std::move(empty);
                h->have_master = false;
            }
        }
    } catch (const std::bad_alloc&) {
        if (h) free_device(h.get());
        set_error("hmat_build: host allocation failed");
        return HMAT_ENOMEM;
    }
    *out = h.release();
    return HMAT_OK;
}

constexpr int kProductFlags = HMAT_TREE_ORDER | HMAT_TRANSPOSE;

// K^T requested and not yet prepared: prepare it now (allocates and
// synchronises), unless `stream` is being captured into a graph.
static int ensure_transpose(hmat_t h, int flags, void* stream, const char* who) {
    if (!(flags & HMAT_TRANSPOSE)) return HMAT_OK;
    hmat_s* own = h->base ? h->base : h;
    if (own->t_ready) return HMAT_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusNone;
    }
    if (cs != cudaStreamCaptureStatusNone) {
        set_error("%s: HMAT_TRANSPOSE during a stream capture needs hmat_prepare_transpose first", who);
        return HMAT_EUNSUPPORTED;
    }
    return prepare_transpose(own);
}

static int matvec_device(hmat_t h, const void* x, void* y, int nrhs, int64_t ldx, int64_t ldy,
                         int flags, void* stream) {
    const Geometry& g = h->geo;
    MatvecArgs a;
    fill_args(h, flags, a);
    a.ldx = ldx;
    a.ldy = ldy;
    a.T = h->dT;
    a.cnt = h->dcnt;
    const int kmax = std::min(h->opts.max_nrhs, max_pass_rhs(h->store));
    // standard admissibility: the streamed kernels, one right-hand side per pass
    const int pass = g.adm ? 1 : choose_pass(a, std::min(nrhs, kmax));
    if (pass <= 0) {
        set_error("hmat_matvec: geometry does not fit the kernels' shared-memory staging");
        return HMAT_EUNSUPPORTED;
    }
    a.kc = pass;
    const size_t eb = vec_elem_bytes(h);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned path = 0;
    for (int c0 = 0; c0 < nrhs; c0 += pass) {
        a.k = std::min(pass, nrhs - c0);
        a.x = static_cast<const char*>(x) + (size_t)c0 * eb;
        a.y = static_cast<char*>(y) + (size_t)c0 * eb;
        for (int which = 0; which < 2; ++which) {
            if (which == 0 && g.nf == 0) continue;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (h->prof) {
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                cudaEventRecord(e0, st);
            }
            const int e = launch_kernel(which, a, stream, &path);
            h->last_path = path;
            if (h->prof) {
                cudaEventRecord(e1, st);
                h->prof_ev[which].emplace_back(e0, e1);
            }
            if (e != 0) {
                set_error("hmat_matvec: launch failed: %s", cudaGetErrorString((cudaError_t)e));
                return HMAT_ECUDA;
            }
        }
    }
    return HMAT_OK;
}

int hmat_matvec(hmat_t h, const void* x, void* y, int nrhs, int64_t ldx, int64_t ldy,
                int flags, void* stream) {
    if (!h || !x || !y) { set_error("hmat_matvec: null pointer"); return HMAT_EINVAL; }
    if (nrhs < 1 || ldx < nrhs || ldy < nrhs) { set_error("hmat_matvec: bad nrhs / leading dimension"); return HMAT_EINVAL; }
    if (flags & ~kProductFlags) { set_error("hmat_matvec: unknown flags"); return HMAT_EINVAL; }
    if (!h->on_device) { set_error("hmat_matvec: handle was built on the host only"); return HMAT_EUNSUPPORTED; }
    if (x == y) { set_error("hmat_matvec: x and y must not overlap"); return HMAT_EINVAL; }
    cudaError_t e = cudaSetDevice(h->opts.device);
    if (e != cudaSuccess) { set_error("cudaSetDevice: %s", cudaGetErrorString(e)); return HMAT_ECUDA; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool cap = false;
    int rc = ensure_transpose(h, flags, stream, "hmat_matvec");
    if (rc) return rc;
    rc = claim_stream(h, st, &cap, "hmat_matvec");
    if (rc) return rc;
    rc = matvec_device(h, x, y, nrhs, ldx, ldy, flags, stream);
    if (rc == HMAT_OK) release_stream(h, st, cap);
    return rc;
}

int hmat_gemv(hmat_t h, double alpha, const void* x, double beta, void* y, int nrhs, int64_t ldx,
              int64_t ldy, int flags, void* stream) {
    if (!h || !x || !y) { set_error("hmat_gemv: null pointer"); return HMAT_EINVAL; }
    if (nrhs < 1 || ldx < nrhs || ldy < nrhs) { set_error("hmat_gemv: bad nrhs / leading dimension"); return HMAT_EINVAL; }
    if (flags & ~kProductFlags) { set_error("hmat_gemv: unknown flags"); return HMAT_EINVAL; }
    if (!std::isfinite(alpha) || !std::isfinite(beta)) { set_error("hmat_gemv: alpha and beta must be finite"); return HMAT_EINVAL; }
    if (!h->on_device) { set_error("hmat_gemv: handle was built on the host only"); return HMAT_EUNSUPPORTED; }
    if (x == y) { set_error("hmat_gemv: x and y must not overlap"); return HMAT_EINVAL; }
    CU_TRY(cudaSetDevice(h->opts.device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool cap = false;
    int rc = ensure_transpose(h, flags, stream, "hmat_gemv");
    if (rc) return rc;
    rc = claim_stream(h, st, &cap, "hmat_gemv");
    if (rc) return rc;
    const size_t eb = vec_elem_bytes(h);
    const int chunk = h->opts.max_nrhs;
    for (int c0 = 0; c0 < nrhs; c0 += chunk) {
        // H x of up to max_nrhs columns into the handle's staging, then
        // y = alpha (H x) + beta y on those columns
        const int kc = std::min(chunk, nrhs - c0);
        rc = matvec_device(h, static_cast<const char*>(x) + (size_t)c0 * eb, h->dY, kc, ldx, kc, flags,
                           stream);
        if (rc) return rc;
        const int e = axpby(h->store == ST_F64, h->tree.N, kc, alpha, h->dY, kc, beta,
                            static_cast<char*>(y) + (size_t)c0 * eb, ldy, stream);
        if (e != 0) {
            set_error("hmat_gemv: launch failed: %s", cudaGetErrorString((cudaError_t)e));
            return HMAT_ECUDA;
        }
    }
    release_stream(h, st, cap);
    return HMAT_OK;
}

int hmat_matvec_host(hmat_t h, const void* x_host, void* y_host, int nrhs, int64_t ldx,
                     int64_t ldy, int flags, void* stream) {
    if (!h || !x_host || !y_host) { set_error("hmat_matvec_host: null pointer"); return HMAT_EINVAL; }
    if (nrhs < 1 || ldx < nrhs || ldy < nrhs) { set_error("hmat_matvec_host: bad nrhs / leading dimension"); return HMAT_EINVAL; }
    if (!h->on_device) { set_error("hmat_matvec_host: handle was built on the host only"); return HMAT_EUNSUPPORTED; }
    if (nrhs > h->opts.max_nrhs) { set_error("hmat_matvec_host: nrhs > max_nrhs"); return HMAT_EUNSUPPORTED; }
    if (flags & ~kProductFlags) { set_error("hmat_matvec_host: unknown flags"); return HMAT_EINVAL; }
    CU_TRY(cudaSetDevice(h->opts.device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool cap = false;
    int rc = ensure_transpose(h, flags, stream, "hmat_matvec_host");
    if (rc) return rc;
    rc = claim_stream(h, st, &cap, "hmat_matvec_host");
    if (rc) return rc;
    const size_t eb = vec_elem_bytes(h);
    const int64_t N = h->tree.N;
    // contiguous vectors (ld == nrhs): one linear copy each way; otherwise
    // one strided 2D copy of N rows of nrhs elements
    const size_t row = (size_t)nrhs * eb;
    if (ldx == nrhs)
        CU_TRY(cudaMemcpyAsync(h->dX, x_host, row * (size_t)N, cudaMemcpyHostToDevice, st));
    else
        CU_TRY(cudaMemcpy2DAsync(h->dX, row, x_host, (size_t)ldx * eb, row, (size_t)N,
                                 cudaMemcpyHostToDevice, st));
    rc = matvec_device(h, h->dX, h->dY, nrhs, nrhs, nrhs, flags, stream);
    if (rc) return rc;
    if (ldy == nrhs)
        CU_TRY(cudaMemcpyAsync(y_host, h->dY, row * (size_t)N, cudaMemcpyDeviceToHost, st));
    else
        CU_TRY(cudaMemcpy2DAsync(y_host, (size_t)ldy * eb, h->dY, row, row, (size_t)N,
                                 cudaMemcpyDeviceToHost, st));
    // the status word rides behind y on the same stream: one synchronisation
    CU_TRY(cudaMemcpyAsync(h->hstatus, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost, st));
    release_stream(h, st, cap);
    CU_TRY(cudaStreamSynchronize(st));
    const int v = *h->hstatus;
    if (v != 0) {
        CU_TRY(cudaMemset(h->dstatus, 0, sizeof(int)));
        set_error("hmat_check: a bounded device-side wait gave up (status word %d)", v);
        return HMAT_ETIMEOUT;
    }
    return HMAT_OK;
}

int hmat_prepare_transpose(hmat_t h) {
    if (!h) { set_error("hmat_prepare_transpose: null handle"); return HMAT_EINVAL; }
    if (!h->on_device) { set_error("hmat_prepare_transpose: handle was built on the host only"); return HMAT_EUNSUPPORTED; }
    return prepare_transpose(h->base ? h->base : h);
}

int64_t hmat_inject_alloc_failure(int64_t after) {
    return g_fail_after.exchange(after < 0 ? -1 : after);
}

int hmat_last_path(hmat_t h) {
    if (!h) { set_error("hmat_last_path: null handle"); return HMAT_EINVAL; }
    return (int)h->last_path;
}

int64_t hmat_launch_count(void) { return hm::launch_count(); }

int hmat_check(hmat_t h, void* stream, int* code) {
    if (code) *code = 0;
    if (!h) { set_error("hmat_check: null handle"); return HMAT_EINVAL; }
    if (!h->on_device || !h->dstatus) return HMAT_OK;
    CU_TRY(cudaSetDevice(h->opts.device));
    CU_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int v = 0;
    CU_TRY(cudaMemcpy(&v, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost));
    if (code) *code = v;
    if (v != 0) {
        CU_TRY(cudaMemset(h->dstatus, 0, sizeof(int)));
        set_error("hmat_check: a bounded device-side wait gave up (status word %d)", v);
        return HMAT_ETIMEOUT;
    }
    return HMAT_OK;
}

int hmat_selftest_timeout(hmat_t h, int limit_us, void* stream, int* code) {
    if (code) *code = 0;
    if (!h) { set_error("hmat_selftest_timeout: null handle"); return HMAT_EINVAL; }
    if (limit_us < 1 || limit_us > 1000000) { set_error("hmat_selftest_timeout: limit_us out of range"); return HMAT_EINVAL; }
    if (!h->on_device || !h->dstatus) { set_error("hmat_selftest_timeout: handle was built on the host only"); return HMAT_EUNSUPPORTED; }
    CU_TRY(cudaSetDevice(h->opts.device));
    const int e = wait_selftest(h->dstatus, (uint64_t)limit_us * 1000ull, stream);
    if (e != 0) { set_error("hmat_selftest_timeout: launch failed: %s", cudaGetErrorString((cudaError_t)e)); return HMAT_ECUDA; }
    return hmat_check(h, stream, code);
}

int hmat_matvec_noalloc(hmat_t h, const void* x, void* y, int nrhs, int64_t ldx, int64_t ldy,
                        int flags, void* stream) {
    if (!h || !x || !y) { set_error("hmat_matvec_noalloc: null pointer"); return HMAT_EINVAL; }
    if (nrhs < 1 || ldx < nrhs || ldy < nrhs) { set_error("hmat_matvec_noalloc: bad nrhs / leading dimension"); return HMAT_EINVAL; }
    if (flags & ~kProductFlags) { set_error("hmat_matvec_noalloc: unknown flags"); return HMAT_EINVAL; }
    if (!h->on_device) { set_error("hmat_matvec_noalloc: handle was built on the host only"); return HMAT_EUNSUPPORTED; }
    if (x == y) { set_error("hmat_matvec_noalloc: x and y must not overlap"); return HMAT_EINVAL; }
    if ((flags & HMAT_TRANSPOSE) && !(h->base ? h->base : h)->t_ready) {
        set_error("hmat_matvec_noalloc: HMAT_TRANSPOSE needs hmat_prepare_transpose first (it allocates)");
        return HMAT_EUNSUPPORTED;
    }
    if (h->geo.adm) {
        set_error("hmat_matvec_noalloc: standard admissibility runs on the streamed kernels only");
        return HMAT_EUNSUPPORTED;
    }
    cudaError_t ce = cudaSetDevice(h->opts.device);
    if (ce != cudaSuccess) { set_error("cudaSetDevice: %s", cudaGetErrorString(ce)); return HMAT_ECUDA; }
    void* scratch = nullptr;
    const int se = static_scratch_address(h->opts.device, &scratch);
    if (se != 0) {
        set_error("hmat_matvec_noalloc: cudaGetSymbolAddress failed: %s",
                  cudaGetErrorString((cudaError_t)se));
        return HMAT_ECUDA;
    }
    const Geometry& g = h->geo;
    MatvecArgs a;
    fill_args(h, flags, a);
    a.ldx = ldx;
    a.ldy = ldy;
    // CUDA-core kernels only: the tensor-core path would use handle-owned
    // prepared operands and status word
    a.status = nullptr;
    a.xprep = a.xprep_lo = a.ttprep = a.ttprep_lo = nullptr;
    // layout inside the static array: [partial sums | arrival counters]
    const size_t acc_bytes = h->store == ST_F64 ? 8 : 4;
    const size_t per_rhs = (size_t)std::max<int64_t>(1, g.t_per_rhs) * acc_bytes;
    const size_t cnt_bytes = ((size_t)std::max<int64_t>(1, g.counters) * sizeof(int) + 255) / 256 * 256;
    if (per_rhs + cnt_bytes > kStaticScratchBytes) {
        set_error("hmat_matvec_noalloc: this H-matrix needs %zu bytes of scratch for one "
                  "right-hand side; the static array holds %zu bytes (use hmat_matvec)",
                  per_rhs + cnt_bytes, (size_t)kStaticScratchBytes);
        return HMAT_EUNSUPPORTED;
    }
    int pass = pass_width(a, std::min(nrhs, max_pass_rhs(h->store)));
    while (pass > 1 && per_rhs * (size_t)pass + cnt_bytes > kStaticScratchBytes) pass /= 2;
    if (pass <= 0) {
        set_error("hmat_matvec_noalloc: geometry does not fit the kernels' shared-memory staging");
        return HMAT_EUNSUPPORTED;
    }
    a.T = scratch;
    a.cnt = reinterpret_cast<int*>(static_cast<char*>(scratch) + kStaticScratchBytes - cnt_bytes);
    // the counters must start at zero; the array may hold another call's data
    ce = cudaMemsetAsync(a.cnt, 0, cnt_bytes, static_cast<cudaStream_t>(stream));
    if (ce != cudaSuccess) {
        set_error("hmat_matvec_noalloc: cudaMemsetAsync: %s", cudaGetErrorString(ce));
        return HMAT_ECUDA;
    }
    a.kc = pass;
    const size_t eb = vec_elem_bytes(h);
    unsigned path = 0;
    for (int c0 = 0; c0 < nrhs; c0 += pass) {
        a.k = std::min(pass, nrhs - c0);
        a.x = static_cast<const char*>(x) + (size_t)c0 * eb;
        a.y = static_cast<char*>(y) + (size_t)c0 * eb;
        for (int which = 0; which < 2; ++which) {
            if (which == 0 && g.nf == 0) continue;
            const int e = launch_kernel(which, a, stream, &path);
            h->last_path = path;
            if (e != 0) {
                set_error("hmat_matvec_noalloc: launch failed: %s", cudaGetErrorString((cudaError_t)e));
                return HMAT_ECUDA;
            }
        }
    }
    return HMAT_OK;
}

int hmat_convert(hmat_t src, int prec, hmat_t* out) {
    if (!src || !out) { set_error("hmat_convert: null pointer"); return HMAT_EINVAL; }
    if (src->base) src = src->base;   // a workspace clone: its base holds the host copy
    if (store_of_prec(prec) < 0) { set_error("hmat_convert: unknown precision"); return HMAT_EINVAL; }
    if (!src->have_master) { set_error("hmat_convert: no host copy (build with keep_host)"); return HMAT_EUNSUPPORTED; }
    if (src->opts.device < 0) { set_error("hmat_convert: source was built on the host only"); return HMAT_EUNSUPPORTED; }
    if (src->tree.m_pad % slot_align(store_of_prec(prec)) != 0) {
        set_error("hmat_convert: leaf slots %d are not a multiple of %d required by precision %d",
                  src->tree.m_pad, slot_align(store_of_prec(prec)), prec);
        return HMAT_EUNSUPPORTED;
    }
    std::unique_ptr<hmat_s> h;
    try {
        h.reset(new hmat_s());
        h->opts = src->opts;
        h->opts.prec = prec;
        h->kernel = src->kernel;
        h->rank = src->rank;
        h->tol = src->tol;
        h->leaf_size = src->leaf_size;
        h->store = store_of_prec(prec);
        h->tree = src->tree;
        h->geo = src->geo;
        h->master = src->master;
        h->have_master = true;
        h->tile_e = src->tile_e;
        const int rc = upload(h.get());
        if (rc) {
            free_device(h.get());
            return rc;
        }
        if (!h->opts.keep_host) {
            Master empty;
            empty.factor_entries = h->master.factor_entries;
            empty.dense_entries = h->master.dense_entries;
            empty.lowrank_blocks = h->master.lowrank_blocks;
            empty.dense_blocks = h->master.dense_blocks;
            h->master = std::move(empty);
            h->have_master = false;
        }
    } catch (const std::bad_alloc&) {
        if (h) free_device(h.get());
        set_error("hmat_convert: host allocation failed");
        return HMAT_ENOMEM;
    }
    *out = h.release();
    return HMAT_OK;
}

// ------------------------------------------------------------ save / load
// Binary file, little-endian: magic "HMATGB3", format version, options,
// kernel / rank / leaf size / tolerance, the tree, the geometry and the
// float64 master factors (the device layout is rebuilt on load).
}  // extern "C"

namespace {
constexpr char kMagic[8] = {'H', 'M', 'A', 'T', 'G', 'B', '3', '\0'};
constexpr uint32_t kFormat = 3;

struct Writer {
    FILE* f;
    bool ok = true;
    void put(const void* p, size_t n) { ok = ok && (n == 0 || fwrite(p, 1, n, f) == n); }
    template <typename T> void pod(const T& v) { put(&v, sizeof(T)); }
    template <typename T> void vec(const std::vector<T>& v) {
        const uint64_t n = v.size();
        pod(n);
        put(v.data(), n * sizeof(T));
    }
};
struct Reader {
    FILE* f;
    bool ok = true;
    void get(void* p, size_t n) { ok = ok && (n == 0 || fread(p, 1, n, f) == n); }
    template <typename T> void pod(T& v) { get(&v, sizeof(T)); }
    template <typename T> void vec(std::vector<T>& v, uint64_t max_n) {
        uint64_t n = 0;
        pod(n);
        if (!ok || n > max_n) { ok = false; return; }
        v.resize(n);
        get(v.data(), n * sizeof(T));
    }
};
}  // namespace

extern "C" {

int hmat_save(hmat_t h, const char* path) {
    if (!h || !path) { set_error("hmat_save: null pointer"); return HMAT_EINVAL; }
    if (h->base) h = h->base;         // a workspace clone: its base holds the host copy
    if (!h->have_master) { set_error("hmat_save: no host copy (build with keep_host or on the host)"); return HMAT_EUNSUPPORTED; }
    FILE* f = fopen(path, "wb");
    if (!f) { set_error("hmat_save: cannot open %s", path); return HMAT_EINVAL; }
    Writer w{f};
    w.put(kMagic, 8);
    w.pod(kFormat);
    w.pod(h->opts);
    w.pod(h->kernel);
    w.pod(h->rank);
    w.pod(h->leaf_size);
    w.pod(h->tol);
    const Tree& t = h->tree;
    w.pod(t.d); w.pod(t.L); w.pod(t.leaf_size); w.pod(t.N); w.pod(t.m_pad); w.pod(t.Np);
    w.vec(t.perm);
    const uint64_t nl = t.beg.size();
    w.pod(nl);
    for (uint64_t l = 0; l < nl; ++l) {
        w.vec(t.beg[l]);
        w.vec(t.cnt[l]);
    }
    w.vec(t.slot);
    w.vec(t.slot_src);
    const Geometry& g = h->geo;
    w.pod(g.d); w.pod(g.s); w.pod(g.L); w.pod(g.nf); w.pod(g.m_pad);
    w.pod(g.Np); w.pod(g.G); w.pod(g.groups); w.pod(g.tile_p); w.pod(g.fac_entries);
    w.pod(g.dense_entries); w.pod(g.t_per_rhs); w.pod(g.counters);
    w.pod(g.adm); w.pod(g.nnb);
    w.vec(g.lv);
    const Master& m = h->master;
    w.pod(m.factor_entries); w.pod(m.dense_entries); w.pod(m.lowrank_blocks); w.pod(m.dense_blocks);
    w.vec(m.U);
    w.vec(m.V);
    w.vec(m.D);
    const bool ok = w.ok && fclose(f) == 0;
    if (!ok) { set_error("hmat_save: write to %s failed", path); return HMAT_EINVAL; }
    return HMAT_OK;
}

int hmat_load(const char* path, const hmat_opts* opts, hmat_t* out) {
    if (!path || !out) { set_error("hmat_load: null pointer"); return HMAT_EINVAL; }
    FILE* f = fopen(path, "rb");
    if (!f) { set_error("hmat_load: cannot open %s", path); return HMAT_EINVAL; }
    std::unique_ptr<hmat_s> h;
    int rc = HMAT_OK;
    try {
        h.reset(new hmat_s());
        Reader r{f};
        char magic[8] = {0};
        uint32_t fmt = 0;
        r.get(magic, 8);
        r.pod(fmt);
        if (!r.ok || std::memcmp(magic, kMagic, 8) != 0 || fmt != kFormat) {
            fclose(f);
            set_error("hmat_load: %s is not an H-matrix file of format %u", path, kFormat);
            return HMAT_EINVAL;
        }
        hmat_opts saved{};
        r.pod(saved);
        r.pod(h->kernel);
        r.pod(h->rank);
        r.pod(h->leaf_size);
        r.pod(h->tol);
        Tree& t = h->tree;
        r.pod(t.d); r.pod(t.L); r.pod(t.leaf_size); r.pod(t.N); r.pod(t.m_pad); r.pod(t.Np);
        const uint64_t big = (uint64_t)1 << 40;
        r.vec(t.perm, big);
        uint64_t nl = 0;
        r.pod(nl);
        if (nl > (uint64_t)kMaxLevels + 1) r.ok = false;
        t.beg.assign(r.ok ? nl : 0, {});
        t.cnt.assign(r.ok ? nl : 0, {});
        for (uint64_t l = 0; r.ok && l < nl; ++l) {
            r.vec(t.beg[l], big);
            r.vec(t.cnt[l], big);
        }
        r.vec(t.slot, big);
        r.vec(t.slot_src, big);
        Geometry& g = h->geo;
        r.pod(g.d); r.pod(g.s); r.pod(g.L); r.pod(g.nf); r.pod(g.m_pad);
        r.pod(g.Np); r.pod(g.G); r.pod(g.groups); r.pod(g.tile_p); r.pod(g.fac_entries);
        r.pod(g.dense_entries); r.pod(g.t_per_rhs); r.pod(g.counters);
        r.pod(g.adm); r.pod(g.nnb);
        r.vec(g.lv, (uint64_t)kMaxLevels + 1);
        Master& m = h->master;
        r.pod(m.factor_entries); r.pod(m.dense_entries); r.pod(m.lowrank_blocks); r.pod(m.dense_blocks);
        r.vec(m.U, big);
        r.vec(m.V, big);
        r.vec(m.D, big);
        fclose(f);
        // consistency of what was read
        const bool sane = r.ok && t.N >= 1 && (t.d == 2 || t.d == 3) && g.d == t.d &&
                          (int64_t)t.perm.size() == t.N && (int64_t)t.slot.size() == t.N &&
                          (int64_t)t.slot_src.size() == t.Np && g.Np == t.Np && g.nf >= 0 &&
                          (int64_t)g.lv.size() == g.nf + 1 && (int64_t)m.U.size() == g.fac_entries &&
                          (g.adm == 0 || g.adm == 1) && g.nnb >= 1 && g.nnb <= 27 &&
                          (int64_t)m.V.size() == g.fac_entries && (int64_t)m.D.size() == g.dense_entries;
        if (!sane) { set_error("hmat_load: %s is truncated or inconsistent", path); return HMAT_EINVAL; }
        h->opts = opts ? *opts : saved;
        if (opts) {
            // the structure is the saved one; storage and placement are the caller's
            h->opts.method = saved.method;
            h->opts.leaf_lowrank = saved.leaf_lowrank;
            h->opts.oversample = saved.oversample;
            h->opts.power_iters = saved.power_iters;
            h->opts.seed = saved.seed;
            h->opts.admissibility = saved.admissibility;
            h->opts.leaf_slot_multiple = saved.leaf_slot_multiple;
        }
        h->store = store_of_prec(h->opts.prec);
        if (h->store < 0) { set_error("hmat_load: unknown precision"); return HMAT_EINVAL; }
        if (t.m_pad % slot_align(h->store) != 0) {
            set_error("hmat_load: leaf slots %d are not a multiple of %d required by the precision",
                      t.m_pad, slot_align(h->store));
            return HMAT_EUNSUPPORTED;
        }
        h->have_master = true;
        h->tile_e = choose_tile_e(h->geo);
        if (h->opts.device >= 0) {
            rc = upload(h.get());
            if (rc) {
                free_device(h.get());
                return rc;
            }
            if (!h->opts.keep_host) {
                Master empty;
                empty.factor_entries = m.factor_entries;
                empty.dense_entries = m.dense_entries;
                empty.lowrank_blocks = m.lowrank_blocks;
                empty.dense_blocks = m.dense_blocks;
                h->master = std::move(empty);
                h->have_master = false;
            }
        }
    } catch (const std::bad_alloc&) {
        if (h) free_device(h.get());
        set_error("hmat_load: host allocation failed");
        return HMAT_ENOMEM;
    }
    *out = h.release();
    return HMAT_OK;
}

int hmat_destroy(hmat_t h) {
    if (!h) return HMAT_OK;
    const int live = h->clones.load();
    if (live > 0) {
        set_error("hmat_destroy: %d workspace clone(s) still borrow this handle's factors; "
                  "destroy them first", live);
        return HMAT_EINVAL;
    }
    hmat_profile(h, 0);
    if (h->on_device) {
        cudaSetDevice(h->opts.device);
        cudaDeviceSynchronize();
        free_device(h);
    }
    if (h->busy_ev) cudaEventDestroy(h->busy_ev);
    if (h->base) h->base->clones.fetch_sub(1);
    delete h;
    return HMAT_OK;
}

int hmat_clone_workspace(hmat_t src, hmat_t* out) {
    if (!src || !out) { set_error("hmat_clone_workspace: null pointer"); return HMAT_EINVAL; }
    if (!src->on_device) { set_error("hmat_clone_workspace: handle was built on the host only"); return HMAT_EUNSUPPORTED; }
    hmat_s* b = src->base ? src->base : src;
    CU_TRY(cudaSetDevice(b->opts.device));
    std::unique_ptr<hmat_s> c;
    try {
        c.reset(new hmat_s());
        c->opts = b->opts;
        c->kernel = b->kernel;
        c->rank = b->rank;
        c->tol = b->tol;
        c->leaf_size = b->leaf_size;
        c->tree = b->tree;
        c->geo = b->geo;
        c->master.factor_entries = b->master.factor_entries;
        c->master.dense_entries = b->master.dense_entries;
        c->master.lowrank_blocks = b->master.lowrank_blocks;
        c->master.dense_blocks = b->master.dense_blocks;
        c->have_master = false;
        c->store = b->store;
        c->tile_e = b->tile_e;
        // borrowed: factors, scales, slot maps, tensor maps and their layout
        c->base = b;
        c->dU = b->dU;
        c->dV = b->dV;
        c->dD = b->dD;
        c->dU_lo = b->dU_lo;
        c->dV_lo = b->dV_lo;
        c->dD_lo = b->dD_lo;
        c->dscU = b->dscU;
        c->dscV = b->dscV;
        c->dscD = b->dscD;
        c->sc_off = b->sc_off;
        c->d_map_orig = b->d_map_orig;
        c->d_map_tree = b->d_map_tree;
        c->dtmaps = b->dtmaps;
        c->tma_rb = b->tma_rb;
        c->tma_rb_u = b->tma_rb_u;
        c->tma_rb_d = b->tma_rb_d;
        c->tc_maps = b->tc_maps;
        c->fp8_maps = b->fp8_maps;
        c->tt_off = b->tt_off;
        c->d_stencil = b->d_stencil;
        c->device_bytes = b->device_bytes;
        int64_t ws = 0;
        const int rc = alloc_workspace(c.get(), ws);
        if (rc) {
            free_device(c.get());
            return rc;
        }
        c->workspace_bytes = ws;
        c->on_device = true;
    } catch (const std::bad_alloc&) {
        if (c) free_device(c.get());
        set_error("hmat_clone_workspace: host allocation failed");
        return HMAT_ENOMEM;
    }
    b->clones.fetch_add(1);
    *out = c.release();
    return HMAT_OK;
}

}  // extern "C"

struct hmat_batch_s {
    int device = 0, store = 0, count = 0;
    int flags = 0;                  // HMAT_TREE_ORDER or 0
    int schedule = HMAT_BATCH_QUEUE;
    int grid_div = 1;               // queue: persistent CTAs per launch = full occupancy / grid_div
    int coarse = 0;                 // queue: right-hand-side widths rounded up to 1, 4, 16, 64
    int branches = 0;               // branch schedule: parallel branches of the graph
    std::vector<hmat_t> hs;
    std::vector<int> nrhs;
    int* d_status = nullptr;        // the plan's status word (refused tasks)
    // queue schedule
    MatvecArgs* d_args = nullptr;
    int* d_units = nullptr;
    void** d_ptrs = nullptr;        // [xs | ys]
    BatchTask* d_tasks = nullptr;
    int ntasks = 0;
    int* d_queues = nullptr;
    void** h_ptrs = nullptr;        // pinned staging of the pointers
    cudaEvent_t ptr_done = nullptr;
    bool ptr_pending = false;
    struct Launch {
        int which, kc;
        BatchLaunch b;
    };
    std::vector<Launch> launches;
    int nqueues = 0;
    // branch schedule: instances in launch order with their branch, the
    // pointers the recorded graph holds, the branch streams and events
    std::vector<int> order, branch_of;
    std::vector<const void*> cap_x;
    std::vector<void*> cap_y;
    std::vector<cudaStream_t> bst;
    std::vector<cudaEvent_t> bev;   // [fork | one join per branch]
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void batch_free(hmat_batch_s* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->ptr_pending && b->ptr_done) cudaEventSynchronize(b->ptr_done);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t s : b->bst)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->bev)
        if (e) cudaEventDestroy(e);
    if (b->ptr_done) cudaEventDestroy(b->ptr_done);
    void* dptrs[] = {b->d_args, b->d_units, b->d_ptrs, b->d_tasks, b->d_queues, b->d_status};
    for (void* p : dptrs)
        if (p) cudaFree(p);
    if (b->h_ptrs) cudaFreeHost(b->h_ptrs);
    delete b;
}

// enqueue every launch of the queue plan on `st` (queues are reset first)
int batch_enqueue(hmat_batch_s* b, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b->d_queues, 0, sizeof(int) * (size_t)b->nqueues, st);
    if (e != cudaSuccess) return (int)e;
    for (const auto& L : b->launches) {
        const int rc = batch_launch(L.which, b->store, L.kc, L.b, st, 0);
        if (rc) return rc;
    }
    return 0;
}

// Bytes one product of instance h with k right-hand sides moves (factors,
// dense blocks, x and y): the weight of the branch schedule's dealing.
double instance_bytes(const hmat_s* h, int k) {
    const int parts = h->store == ST_BF16X2 ? 2 : 1;
    const double es = factor_elem_bytes(h->store) * parts;
    const double esd = h->store == ST_FP8 ? 2.0 : es;
    return 2.0 * (double)h->geo.fac_entries * es + (double)h->geo.dense_entries * esd +
           2.0 * (double)h->tree.N * k * (double)vec_elem_bytes(h);
}

// Records the branch schedule's graph for the pointers xs / ys: every
// instance's own product on its branch, the branches forked from and
// joined to the capture stream.
int batch_record(hmat_batch_s* b, const void* const* xs, void* const* ys) {
    cudaError_t ce = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
    if (ce != cudaSuccess) { set_error("hmat_batch_matvec: capture: %s", cudaGetErrorString(ce)); return HMAT_ECUDA; }
    int rc = HMAT_OK;
    ce = cudaEventRecord(b->bev[0], b->cap);
    for (int j = 0; j < b->branches && ce == cudaSuccess; ++j) ce = cudaStreamWaitEvent(b->bst[j], b->bev[0], 0);
    if (ce != cudaSuccess) rc = HMAT_ECUDA;
    for (size_t q = 0; q < b->order.size() && !rc; ++q) {
        const int i = b->order[q];
        const int k = b->nrhs[i];
        rc = matvec_device(b->hs[i], xs[i], ys[i], k, k, k, b->flags, b->bst[b->branch_of[i]]);
    }
    // every branch joins the capture stream, also after a failure, so that
    // ending the capture releases all of them
    for (int j = 0; j < b->branches; ++j) {
        cudaError_t je = cudaEventRecord(b->bev[1 + j], b->bst[j]);
        if (je == cudaSuccess) je = cudaStreamWaitEvent(b->cap, b->bev[1 + j], 0);
        if (je != cudaSuccess && !rc) {
            ce = je;
            rc = HMAT_ECUDA;
        }
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
    if (!rc && ee != cudaSuccess) rc = HMAT_ECUDA;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        if (ce != cudaSuccess || ee != cudaSuccess)
            set_error("hmat_batch_matvec: graph capture failed: %s",
                      cudaGetErrorString(ce != cudaSuccess ? ce : ee));
        return rc;
    }
    // the executable graph is updated in place when the topology allows
    bool updated = false;
    if (b->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(b->exec, g, &info) == cudaSuccess) {
            updated = true;
        } else {
            cudaGetLastError();
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
    }
    if (!updated) {
        ce = cudaGraphInstantiate(&b->exec, g, 0);
        if (ce != cudaSuccess) {
            cudaGraphDestroy(g);
            b->exec = nullptr;
            set_error("hmat_batch_matvec: graph instantiation failed: %s", cudaGetErrorString(ce));
            return HMAT_ECUDA;
        }
    }
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph = g;
    b->cap_x.assign(xs, xs + b->count);
    b->cap_y.assign(ys, ys + b->count);
    return HMAT_OK;
}

// Branch schedule: the instances dealt largest first (by bytes) to the
// least loaded of `branches` branches; streams and events for the capture.
int batch_build_branches(hmat_batch_s* b, int branches) {
    b->branches = std::max(1, std::min(branches, b->count));
    std::vector<std::pair<double, int>> w(b->count);
    for (int i = 0; i < b->count; ++i) w[i] = {instance_bytes(b->hs[i], b->nrhs[i]), i};
    std::stable_sort(w.begin(), w.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    std::vector<double> load(b->branches, 0.0);
    b->branch_of.assign(b->count, 0);
    for (const auto& e : w) {
        const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->branch_of[e.second] = j;
        load[j] += e.first;
    }
    // launch order: branch by branch, largest first within a branch
    for (int j = 0; j < b->branches; ++j)
        for (const auto& e : w)
            if (b->branch_of[e.second] == j) b->order.push_back(e.second);
    cudaError_t ce = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    b->bst.assign(b->branches, nullptr);
    b->bev.assign(b->branches + 1, nullptr);
    for (int j = 0; j < b->branches && ce == cudaSuccess; ++j)
        ce = cudaStreamCreateWithFlags(&b->bst[j], cudaStreamNonBlocking);
    for (size_t j = 0; j < b->bev.size() && ce == cudaSuccess; ++j)
        ce = cudaEventCreateWithFlags(&b->bev[j], cudaEventDisableTiming);
    if (ce != cudaSuccess) { set_error("hmat_batch_create: %s", cudaGetErrorString(ce)); return HMAT_ECUDA; }
    return HMAT_OK;
}

}  // namespace

namespace {

// Build a plan with a given schedule: the queue (grid divisor, width
// grouping) or `branches` parallel branches.
int batch_build(const hmat_t* hs, int count, const int* nrhs, int flags, int schedule, int grid_div,
                int coarse, int branches, hmat_batch_t* out) {
    if (!hs || !nrhs || !out || count < 1) { set_error("hmat_batch_create: bad arguments"); return HMAT_EINVAL; }
    if (flags & ~HMAT_TREE_ORDER) { set_error("hmat_batch_create: unknown flags"); return HMAT_EINVAL; }
    for (int i = 0; i < count; ++i) {
        if (!hs[i] || !hs[i]->on_device) { set_error("hmat_batch_create: handle %d is not on a device", i); return HMAT_EINVAL; }
        if (hs[i]->opts.device != hs[0]->opts.device || hs[i]->store != hs[0]->store) {
            set_error("hmat_batch_create: handles must share the device and the precision");
            return HMAT_EUNSUPPORTED;
        }
        if (nrhs[i] < 1) { set_error("hmat_batch_create: nrhs[%d] < 1", i); return HMAT_EINVAL; }
        if (hs[i]->geo.adm) {
            set_error("hmat_batch_create: handle %d uses standard admissibility (streamed kernels only)", i);
            return HMAT_EUNSUPPORTED;
        }
    }
    {
        // one product at a time per workspace: no handle twice
        std::vector<hmat_t> sorted(hs, hs + count);
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
            set_error("hmat_batch_create: a handle appears twice (use hmat_clone_workspace handles)");
            return HMAT_EINVAL;
        }
    }
    hmat_batch_s* b = new hmat_batch_s();
    b->device = hs[0]->opts.device;
    b->store = hs[0]->store;
    b->count = count;
    b->flags = flags;
    b->schedule = schedule;
    b->grid_div = grid_div;
    b->coarse = coarse;
    b->hs.assign(hs, hs + count);
    b->nrhs.assign(nrhs, nrhs + count);
    cudaError_t ce = cudaSetDevice(b->device);
    if (ce != cudaSuccess) { batch_free(b); set_error("cudaSetDevice: %s", cudaGetErrorString(ce)); return HMAT_ECUDA; }
    int64_t dummy = 0;
    int rc = dev_alloc((void**)&b->d_status, sizeof(int), dummy);
    if (!rc && cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess) rc = HMAT_ECUDA;
    if (rc) { batch_free(b); return rc; }
    std::vector<MatvecArgs> args(count);
    std::vector<int> units(count, 0), ptiles(count, 0), etiles(count, 0);
    std::vector<size_t> psm(count, 0), esm(count, 0);
    for (int i = 0; i < count; ++i) {
        hmat_s* h = hs[i];
        MatvecArgs& a = args[i];
        fill_args(h, flags, a);
        a.T = h->dT;
        a.cnt = h->dcnt;
        const int kmax = std::min(h->opts.max_nrhs, max_pass_rhs(h->store));
        const int kalloc = workspace_width(h);
        int kc = schedule == HMAT_BATCH_BRANCHES ? choose_pass(a, nrhs[i]) : pass_width(a, nrhs[i]);
        if (coarse && schedule == HMAT_BATCH_QUEUE) {
            // fewer width classes (fewer launches, more idle lanes)
            const int want = nrhs[i] <= 1 ? 1 : nrhs[i] <= 4 ? 4 : nrhs[i] <= 16 ? 16 : 64;
            const int kw = pass_width(a, want);
            if (kw >= nrhs[i] && kw <= kalloc) kc = kw;
        }
        if (kc < nrhs[i] || kc > kalloc || nrhs[i] > kmax) {
            batch_free(b);
            set_error("hmat_batch_create: instance %d: %d right-hand sides need more than one pass",
                      i, nrhs[i]);
            return HMAT_EUNSUPPORTED;
        }
        if (schedule == HMAT_BATCH_BRANCHES) continue;
        a.kc = kc;
        a.k = nrhs[i];
        a.ldx = a.ldy = nrhs[i];
        a.x = nullptr;
        a.y = nullptr;
        int u = 0;
        rc = batch_setup(a, 0, &u, &psm[i]);
        units[i] = u;
        ptiles[i] = a.nf > 0 ? (int)(a.Np / a.tile_p) : 0;
        if (!rc) rc = batch_setup(a, 1, &etiles[i], &esm[i]);
        if (rc) { batch_free(b); set_error("hmat_batch_create: setup failed"); return HMAT_ECUDA; }
    }
    if (schedule == HMAT_BATCH_BRANCHES) {
        rc = batch_build_branches(b, branches);
        if (rc) { batch_free(b); return rc; }
        *out = b;
        return HMAT_OK;
    }
    // group by compiled width; tasks of a launch sorted largest first
    std::vector<int> widths;
    for (int i = 0; i < count; ++i)
        if (std::find(widths.begin(), widths.end(), args[i].kc) == widths.end()) widths.push_back(args[i].kc);
    std::sort(widths.begin(), widths.end());
    struct Pending { int which, kc; std::vector<BatchTask> tasks; size_t smem; };
    std::vector<Pending> pend;
    for (int which = 0; which < 2; ++which)
        for (int kc : widths) {
            Pending P{which, kc, {}, 0};
            std::vector<std::pair<double, BatchTask>> cost;
            for (int i = 0; i < count; ++i) {
                if (args[i].kc != kc) continue;
                const MatvecArgs& a = args[i];
                double cols = 0;
                for (int l = 1; l <= a.nf; ++l) cols += (double)a.s * a.lv[l].r;
                const int nt = which == 0 ? ptiles[i] : etiles[i];
                const double c = which == 0 ? (double)a.tile_p * cols
                                            : (double)a.tile_e * (cols + (double)a.G);
                for (int t = 0; t < nt; ++t) cost.push_back({c, BatchTask{i, t}});
                P.smem = std::max(P.smem, which == 0 ? psm[i] : esm[i]);
            }
            std::stable_sort(cost.begin(), cost.end(),
                             [](const auto& x, const auto& y) { return x.first > y.first; });
            for (auto& c : cost) P.tasks.push_back(c.second);
            if (!P.tasks.empty()) pend.push_back(std::move(P));
        }
    size_t ntask_total = 0;
    for (auto& P : pend) ntask_total += P.tasks.size();
    b->ntasks = (int)ntask_total;
    if (!rc) rc = dev_alloc((void**)&b->d_args, sizeof(MatvecArgs) * count, dummy);
    if (!rc) rc = dev_alloc((void**)&b->d_units, sizeof(int) * count, dummy);
    if (!rc) rc = dev_alloc((void**)&b->d_ptrs, sizeof(void*) * 2 * count, dummy);
    if (!rc) rc = dev_alloc((void**)&b->d_tasks, sizeof(BatchTask) * std::max<size_t>(1, ntask_total), dummy);
    if (!rc) rc = dev_alloc((void**)&b->d_queues, sizeof(int) * std::max<size_t>(1, pend.size()), dummy);
    if (rc) { batch_free(b); return rc; }
    ce = cudaMallocHost((void**)&b->h_ptrs, sizeof(void*) * 2 * count);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&b->ptr_done, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaMemcpy(b->d_args, args.data(), sizeof(MatvecArgs) * count, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(b->d_units, units.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
    size_t off = 0;
    for (size_t q = 0; q < pend.size() && ce == cudaSuccess; ++q) {
        Pending& P = pend[q];
        ce = cudaMemcpy(b->d_tasks + off, P.tasks.data(), sizeof(BatchTask) * P.tasks.size(),
                        cudaMemcpyHostToDevice);
        hmat_batch_s::Launch L;
        L.which = P.which;
        L.kc = P.kc;
        L.b.args = b->d_args;
        L.b.units = b->d_units;
        L.b.xs = (const void* const*)b->d_ptrs;
        L.b.ys = (void* const*)(b->d_ptrs + count);
        L.b.tasks = b->d_tasks + off;
        L.b.ntasks = (int)P.tasks.size();
        L.b.queue = b->d_queues + q;
        L.b.smem = P.smem;
        L.b.grid_div = grid_div;
        L.b.count = count;
        L.b.status = b->d_status;
        b->launches.push_back(L);
        off += P.tasks.size();
    }
    b->nqueues = (int)pend.size();
    if (ce != cudaSuccess) { batch_free(b); set_error("hmat_batch_create: %s", cudaGetErrorString(ce)); return HMAT_ECUDA; }
    // one CUDA graph: queue reset, the project launches, the expand launches
    ce = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    // kernel attributes are set outside the capture
    for (const auto& L : b->launches) {
        if (ce != cudaSuccess) break;
        const int drc = batch_launch(L.which, b->store, L.kc, L.b, b->cap, 1);
        if (drc) ce = (cudaError_t)drc;
    }
    if (ce == cudaSuccess) ce = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
    if (ce == cudaSuccess) {
        const int erc = batch_enqueue(b, b->cap);
        cudaGraph_t g = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
        b->graph = g;
        ce = erc ? (cudaError_t)erc : ee;
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (ce != cudaSuccess) {
        batch_free(b);
        set_error("hmat_batch_create: graph capture failed: %s", cudaGetErrorString(ce));
        return HMAT_ECUDA;
    }
    *out = b;
    return HMAT_OK;
}

constexpr int kDefaultBranches = 8;

}  // namespace

extern "C" {

int hmat_batch_create(const hmat_t* hs, int count, const int* nrhs, int flags,
                      hmat_batch_t* out) {
    const int sched = flags & (HMAT_BATCH_QUEUE | HMAT_BATCH_BRANCHES);
    if (sched == (HMAT_BATCH_QUEUE | HMAT_BATCH_BRANCHES)) {
        set_error("hmat_batch_create: one schedule at a time");
        return HMAT_EINVAL;
    }
    const int schedule = sched ? sched : HMAT_BATCH_QUEUE;
    return batch_build(hs, count, nrhs, flags & ~sched, schedule, 1, 0, kDefaultBranches, out);
}

int hmat_batch_autotune(hmat_batch_t b, const void* const* xs, void* const* ys, void* stream, int reps,
                        hmat_batch_tuning* out) {
    if (!b || !xs || !ys || reps < 1) { set_error("hmat_batch_autotune: bad arguments"); return HMAT_EINVAL; }
    CU_TRY(cudaSetDevice(b->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    struct Cand { int schedule, div, coarse, branches; };
    std::vector<Cand> cands;
    for (int coarse = 0; coarse < 2; ++coarse)
        for (int div : {1, 2, 4}) cands.push_back({HMAT_BATCH_QUEUE, div, coarse, 0});
    for (int br : {4, 8, 16, 32})
        if (br <= b->count || br == 4) cands.push_back({HMAT_BATCH_BRANCHES, 1, 0, br});
    double best = -1.0, dflt = -1.0, bq = -1.0, bb = -1.0;
    Cand win{b->schedule, b->grid_div, b->coarse, b->branches};
    int tried = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU_TRY(cudaEventCreate(&e0));
    CU_TRY(cudaEventCreate(&e1));
    int rc = HMAT_OK;
    for (const Cand& c : cands) {
        hmat_batch_t p = nullptr;
        rc = batch_build(b->hs.data(), b->count, b->nrhs.data(), b->flags, c.schedule, c.div, c.coarse,
                         c.branches, &p);
        if (rc) break;
        rc = hmat_batch_matvec(p, xs, ys, stream);           // warm-up (records the branch graph)
        float ms = 0.f;
        if (!rc && cudaEventRecord(e0, st) != cudaSuccess) rc = HMAT_ECUDA;
        for (int r = 0; r < reps && !rc; ++r) rc = hmat_batch_matvec(p, xs, ys, stream);
        if (!rc && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = HMAT_ECUDA;
        if (!rc) {
            const double t = (double)ms / reps;
            const bool is_default = c.schedule == b->schedule &&
                                    (c.schedule == HMAT_BATCH_QUEUE ? (c.div == 1 && c.coarse == 0)
                                                                    : c.branches == kDefaultBranches);
            if (is_default) dflt = t;
            double& bs = c.schedule == HMAT_BATCH_QUEUE ? bq : bb;
            if (bs < 0 || t < bs) bs = t;
            if (best < 0 || t < best) {
                best = t;
                win = c;
            }
            ++tried;
        }
        cudaStreamSynchronize(st);
        batch_free(p);
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (win.schedule != b->schedule || win.div != b->grid_div || win.coarse != b->coarse ||
        win.branches != b->branches) {
        hmat_batch_t nb = nullptr;
        rc = batch_build(b->hs.data(), b->count, b->nrhs.data(), b->flags, win.schedule, win.div, win.coarse,
                         win.branches, &nb);
        if (rc) return rc;
        if (b->ptr_pending) CU_TRY(cudaEventSynchronize(b->ptr_done));
        std::swap(*b, *nb);
        batch_free(nb);
    }
    // the outputs are those of the chosen schedule
    rc = hmat_batch_matvec(b, xs, ys, stream);
    if (rc) return rc;
    CU_TRY(cudaStreamSynchronize(st));
    if (out) {
        out->grid_div = win.schedule == HMAT_BATCH_QUEUE ? win.div : 0;
        out->coarse_widths = win.schedule == HMAT_BATCH_QUEUE ? win.coarse : 0;
        out->candidates = tried;
        out->ms = best;
        out->ms_default = dflt;
        out->schedule = win.schedule;
        out->branches = win.schedule == HMAT_BATCH_BRANCHES ? b->branches : 0;
        out->ms_queue = bq;
        out->ms_branches = bb;
    }
    return HMAT_OK;
}

int hmat_batch_matvec(hmat_batch_t b, const void* const* xs, void* const* ys, void* stream) {
    if (!b || !xs || !ys) { set_error("hmat_batch_matvec: null pointer"); return HMAT_EINVAL; }
    for (int i = 0; i < b->count; ++i)
        if (!xs[i] || !ys[i] || xs[i] == ys[i]) { set_error("hmat_batch_matvec: bad x/y of instance %d", i); return HMAT_EINVAL; }
    CU_TRY(cudaSetDevice(b->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (b->schedule == HMAT_BATCH_BRANCHES) {
        bool same = b->exec != nullptr;
        for (int i = 0; i < b->count && same; ++i) same = b->cap_x[i] == xs[i] && b->cap_y[i] == ys[i];
        if (!same) {
            const int rc = batch_record(b, xs, ys);
            if (rc) return rc;
        }
        CU_TRY(cudaGraphLaunch(b->exec, st));
        return HMAT_OK;
    }
    if (b->ptr_pending) CU_TRY(cudaEventSynchronize(b->ptr_done));
    for (int i = 0; i < b->count; ++i) {
        b->h_ptrs[i] = const_cast<void*>(xs[i]);
        b->h_ptrs[b->count + i] = ys[i];
    }
    CU_TRY(cudaMemcpyAsync(b->d_ptrs, b->h_ptrs, sizeof(void*) * 2 * b->count,
                           cudaMemcpyHostToDevice, st));
    CU_TRY(cudaEventRecord(b->ptr_done, st));
    b->ptr_pending = true;
    CU_TRY(cudaGraphLaunch(b->exec, st));
    return HMAT_OK;
}

int hmat_batch_check(hmat_batch_t b, void* stream, int* code) {
    if (code) *code = 0;
    if (!b) { set_error("hmat_batch_check: null plan"); return HMAT_EINVAL; }
    CU_TRY(cudaSetDevice(b->device));
    CU_TRY(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int v = 0;
    CU_TRY(cudaMemcpy(&v, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    int first = v;
    if (v != 0) {
        // a skipped project task leaves its nodes' arrival counters short of
        // their tile count: clear every instance's counters with the word
        CU_TRY(cudaMemset(b->d_status, 0, sizeof(int)));
        for (const hmat_s* h : b->hs)
            if (h->dcnt) CU_TRY(cudaMemset(h->dcnt, 0, (size_t)std::max<int64_t>(1, h->geo.counters) * sizeof(int)));
    }
    bool timeout = false;
    for (int i = 0; i < b->count; ++i) {
        int c = 0;
        const int rc = hmat_check(b->hs[i], stream, &c);
        if (rc == HMAT_ETIMEOUT) {
            timeout = true;
            if (!first) first = c;
        } else if (rc) {
            return rc;
        }
    }
    if (code) *code = first;
    if (v != 0) {
        set_error("hmat_batch_check: a queue kernel refused a task (status word %d)", v);
        return HMAT_EDEVICE;
    }
    if (timeout) {
        set_error("hmat_batch_check: a bounded device-side wait gave up (status word %d)", first);
        return HMAT_ETIMEOUT;
    }
    return HMAT_OK;
}

int hmat_batch_poison_task(hmat_batch_t b, int task, int inst, int tile) {
    if (!b) { set_error("hmat_batch_poison_task: null plan"); return HMAT_EINVAL; }
    if (b->schedule != HMAT_BATCH_QUEUE) { set_error("hmat_batch_poison_task: branch schedule has no task table"); return HMAT_EUNSUPPORTED; }
    if (task < 0 || task >= b->ntasks) { set_error("hmat_batch_poison_task: task out of range"); return HMAT_EINVAL; }
    CU_TRY(cudaSetDevice(b->device));
    CU_TRY(cudaDeviceSynchronize());
    const BatchTask t{inst, tile};
    CU_TRY(cudaMemcpy(b->d_tasks + task, &t, sizeof(t), cudaMemcpyHostToDevice));
    return HMAT_OK;
}

int hmat_batch_destroy(hmat_batch_t b) {
    batch_free(b);
    return HMAT_OK;
}

int hmat_profile(hmat_t h, int enable) {
    if (!h) { set_error("hmat_profile: null handle"); return HMAT_EINVAL; }
    for (int w = 0; w < 2; ++w) {
        for (auto& pr : h->prof_ev[w]) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        h->prof_ev[w].clear();
        h->prof_launches[w] = 0;
        h->prof_ms[w] = 0.0;
    }
    h->prof = enable != 0;
    return HMAT_OK;
}

int hmat_profile_read(hmat_t h, int64_t* launches, double* ms) {
    if (!h || !launches || !ms) { set_error("hmat_profile_read: null pointer"); return HMAT_EINVAL; }
    for (int w = 0; w < 2; ++w) {
        for (auto& pr : h->prof_ev[w]) {
            cudaError_t e = cudaEventSynchronize(pr.second);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pr.first, pr.second);
            if (e != cudaSuccess) {
                set_error("hmat_profile_read: %s", cudaGetErrorString(e));
                return HMAT_ECUDA;
            }
            h->prof_ms[w] += t;
            h->prof_launches[w] += 1;
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        h->prof_ev[w].clear();
        launches[w] = h->prof_launches[w];
        ms[w] = h->prof_ms[w];
    }
    return HMAT_OK;
}

int hmat_info(hmat_t h, hmat_info_t* out) {
    if (!h || !out) { set_error("hmat_info: null pointer"); return HMAT_EINVAL; }
    std::memset(out, 0, sizeof(*out));
    const Geometry& g = h->geo;
    out->N = h->tree.N;
    out->d = g.d;
    out->depth = g.L;
    out->lowrank_levels = g.nf;
    out->leaf_slots = g.m_pad;
    out->prec = h->opts.prec;
    out->padded_N = g.Np;
    out->lowrank_blocks = h->master.lowrank_blocks;
    out->dense_blocks = h->master.dense_blocks;
    out->factor_entries = h->master.factor_entries;
    out->dense_entries = h->master.dense_entries;
    out->device_bytes = h->device_bytes;
    out->workspace_bytes = h->workspace_bytes;
    for (int l = 1; l <= g.nf && l < 32; ++l) out->rank_per_level[l] = g.lv[l].r;
    out->admissibility = g.adm;
    out->partners = g.s;
    out->near_groups = g.nnb;
    return HMAT_OK;
}

int hmat_get_perm(hmat_t h, int64_t* perm) {
    if (!h || !perm) { set_error("hmat_get_perm: null pointer"); return HMAT_EINVAL; }
    std::memcpy(perm, h->tree.perm.data(), sizeof(int64_t) * h->tree.N);
    return HMAT_OK;
}

int hmat_export_block(hmat_t h, int level, int64_t t, int64_t s, double* U, double* V,
                      int64_t* sizes) {
    if (!h) { set_error("hmat_export_block: null handle"); return HMAT_EINVAL; }
    if (h->base) h = h->base;         // a workspace clone: its base holds the host copy
    const Geometry& g = h->geo;
    const Tree& tr = h->tree;
    if (level < 1 || level > g.nf) { set_error("hmat_export_block: level out of range"); return HMAT_EINVAL; }
    const int64_t nodes = (int64_t)1 << (g.d * level);
    const int nc = 1 << g.d;
    int qv = 0, qu = 0;
    if (!g.adm) {
        if (t < 0 || s < 0 || t >= nodes || s >= nodes || t == s || t / nc != s / nc) {
            set_error("hmat_export_block: t, s must be distinct siblings");
            return HMAT_EINVAL;
        }
        const int ci = (int)(t % nc), cj = (int)(s % nc);
        qv = ci < cj ? ci : ci - 1;
        qu = cj < ci ? cj : cj - 1;
    } else {
        // standard admissibility: s must be in t's interaction list
        if (t < 0 || s < 0 || t >= nodes || s >= nodes) {
            set_error("hmat_export_block: node out of range");
            return HMAT_EINVAL;
        }
        Stencil st;
        build_stencil(g.d, st);
        int ct[3], cs[3], dl[3] = {0, 0, 0};
        node_coords(t, g.d, level, ct);
        node_coords(s, g.d, level, cs);
        for (int a = 0; a < g.d; ++a) dl[a] = cs[a] - ct[a];
        qu = stencil_slot(st, ct, dl);
        if (qu < 0) {
            set_error("hmat_export_block: s is not in the interaction list of t");
            return HMAT_EINVAL;
        }
        int p = 0;
        for (int a = 0; a < g.d; ++a) p |= (ct[a] & 1) << a;
        qv = st.rev[(size_t)p * st.nslot + qu];
    }
    const int64_t nt = tr.cnt[level][t], ns = tr.cnt[level][s];
    if (sizes) { sizes[0] = nt; sizes[1] = ns; }
    if (!U && !V) return HMAT_OK;
    if (!h->have_master) { set_error("hmat_export_block: no host copy (keep_host)"); return HMAT_EUNSUPPORTED; }
    const LevelGeom& lg = g.lv[level];
    const int64_t sr = (int64_t)g.s * lg.r;
    for (int c = 0; c < lg.r; ++c) {
        if (U) {
            const double* uc = h->master.U.data() + lg.fac_off + (t * sr + qu * lg.r + c) * lg.n;
            for (int64_t a = 0; a < nt; ++a) U[a * lg.r + c] = uc[tr.slot[tr.beg[level][t] + a] - t * lg.n];
        }
        if (V) {
            const double* vc = h->master.V.data() + lg.fac_off + (s * sr + qv * lg.r + c) * lg.n;
            for (int64_t a = 0; a < ns; ++a) V[a * lg.r + c] = vc[tr.slot[tr.beg[level][s] + a] - s * lg.n];
        }
    }
    return HMAT_OK;
}

int hmat_export_dense(hmat_t h, int64_t gi, double* D, int64_t* size) {
    if (!h) { set_error("hmat_export_dense: null handle"); return HMAT_EINVAL; }
    if (h->base) h = h->base;         // a workspace clone: its base holds the host copy
    const Geometry& g = h->geo;
    const Tree& tr = h->tree;
    if (gi < 0 || gi >= g.groups) { set_error("hmat_export_dense: group out of range"); return HMAT_EINVAL; }
    const int64_t n = tr.cnt[g.nf][gi], b0 = tr.beg[g.nf][gi];
    if (size) *size = n;
    if (!D) return HMAT_OK;
    if (!h->have_master) { set_error("hmat_export_dense: no host copy (keep_host)"); return HMAT_EUNSUPPORTED; }
    // the group's block with itself (standard admissibility: the centre of
    // its 3^d touching source groups)
    const int kc = g.adm ? (g.nnb - 1) / 2 : 0;
    const double* Dg = h->master.D.data() + (gi * g.nnb + kc) * g.G * g.G;
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = 0; b < n; ++b)
            D[a * n + b] = Dg[(tr.slot[b0 + b] - gi * g.G) * g.G + (tr.slot[b0 + a] - gi * g.G)];
    return HMAT_OK;
}

}  // extern "C"

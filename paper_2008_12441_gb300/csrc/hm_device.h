// Device-side parameter blocks and launcher declarations shared by the
// CUDA translation units and the C-ABI glue.
#pragma once
#include <cstdint>

namespace hm {

constexpr int kMaxLevels = 24;

struct DevLevel {
    int r;            // padded rank r_l
    int pad_;
    int64_t n;        // slots per node n_l
    int64_t seg_len;  // min(n_l, project tile)
    int64_t fac_off;  // entry offset of the level in U / V
    int64_t t_off;    // partial-sum offset (units of one rhs)
    int64_t sc_off;   // scale offset of the level (per node-slot or per column)
};

// Storage codes (device factor element types).
enum StoreKind { ST_F64 = 0, ST_F32 = 1, ST_BF16 = 2, ST_BF16X2 = 3, ST_FP8 = 4 };

struct MatvecArgs {
    // geometry
    int d, s, nf, nlev_pad_;
    int64_t Np, G, tile_p;
    DevLevel lv[kMaxLevels + 1];
    // factors (type given by the storage kind)
    const void* U;
    const void* V;
    const void* D;
    const void* U_lo;     // split storage: low parts
    const void* V_lo;
    const void* D_lo;
    const float* scU;     // scales (bf16: per node-slot block; fp8: per column)
    const float* scV;
    const float* scD;     // per group
    // vectors
    const void* x;
    void* y;
    int64_t ldx, ldy;
    const int64_t* map;   // slot -> vector row (or -1); nullptr = identity
    int k;                // right-hand sides in this pass
    int kc;               // rhs stride of the partial-sum buffer
    void* T;              // partial sums (float, or double in the FP64 mode)
    int64_t tile_e;       // expand tile (slots)
};

// Launch kernel `which` (0 = project, Step 1; 1 = expand, Steps 2-5) for one
// pass of a.k <= a.kc right-hand sides.  Returns a cudaError_t value.
int launch_kernel(int which, int store_kind, const MatvecArgs& a, void* stream);
// Maximum right-hand sides per pass supported by the kernels of a storage kind.
int max_pass_rhs(int store_kind);
// Compiled RHS width for a pass of k right-hand sides: the smallest width
// >= k whose shared-memory staging fits, else the widest that fits (0: none).
int pass_width(int store_kind, const MatvecArgs& a, int k);

// Size of the static partial-sum array used by hmat_matvec_noalloc (8 MiB).
constexpr size_t kStaticScratchBytes = (size_t)8 << 20;
// Device address of that array on `device` (which must be current); the
// first call per device looks it up with cudaGetSymbolAddress.  Returns a
// cudaError_t value.
int static_scratch_address(int device, void** ptr);

}  // namespace hm

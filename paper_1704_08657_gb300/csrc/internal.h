// internal.h -- host/device parameter blocks and the launcher interface
// between the C ABI (api.cu) and the kernel translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dwt2 {

// device status word bits
enum : unsigned { DEV_TIMEOUT = 1u, DEV_CHECK = 2u };

enum { SCHEME_NONSEP = 0, SCHEME_REDUCED = 1, SCHEME_SEP = 2, SCHEME_POLYCONV = 3, SCHEME_CONV = 4, SCHEME_NSCONV = 5 };
enum { WAV_CDF97 = 0, WAV_CDF53I = 1, WAV_DD137 = 2 };
enum { DT_F32 = 0, DT_F16 = 1, DT_BF16 = 2, DT_I32 = 3 };

// One forward level.  Input pixels come through the two tensor maps; the
// output is written in Mallat layout: LL to `ll` (compute type when ll_is_ct,
// i.e. an intermediate band in the workspace, else the coefficient type), HL
// to coef[row][wq + j], LH to coef[hq + row][j], HH to coef[hq + row][wq + j].
struct FwdParams {
    int h, w;                  // level input size in pixels (>= 2)
    int hq, wq, hh, wh;        // ceil and floor halves
    int n_strips, seg_rows, n_segs, n_units;
    int balanced;              // 1: each warp takes one contiguous range of strip-major quad rows
    void* coef;                // top-left of the level's region, coefficient type
    int64_t coef_pitch;        // elements
    void* ll;                  // LL destination
    int64_t ll_pitch;
    int ll_is_ct;
    int vec_lo, vec_hi, vec_ll;  // pair-store alignment: LH, HL / HH, LL
    unsigned* status;          // device status word (may be null)
    uint64_t timeout_ns;       // bounded-wait limit
    int pdl;                   // host side: launch as a programmatic dependent of the previous kernel
    // Overlap with the previous level (single-image plans): instead of
    // waiting for the previous grid, a unit waits (bounded) until the previous
    // level's segments covering its input rows are complete, and every unit
    // bumps its own segment's counter after its stores.
    int dep_need, dep_seg;     // strips of a previous-level segment; its height in input rows
    const unsigned* dep_ctr;   // previous level's segment counters (null: wait for the previous grid)
    unsigned* out_ctr;         // this level's segment counters (null: none)
    int test_drop;             // test-only hook: unit (strip 0, segment 0) never bumps its counter
};

// One inverse or adjoint level: bands in, pixels (compute type) out.
struct InvParams {
    int h, w;
    int hq, wq, hh, wh;
    int n_strips, seg_rows, n_segs, n_units;
    int balanced;
    const void* coef;          // detail bands (coefficient type), level origin
    int64_t coef_pitch;
    const void* ll;            // LL band: compute type when ll_is_ct
    int64_t ll_pitch;
    int ll_is_ct;
    void* out;                 // output pixels, compute type
    int64_t out_pitch;
    int vec_in_lo, vec_in_hi, vec_ll, vec_out;
    unsigned* status;
    uint64_t timeout_ns;       // bounded-wait limit
    // adjoint of an L1 loss on the detail bands: band values v read from the
    // coefficients become l1_scale * sign(v) (detail bands) or 0 (coarsest LL);
    // with l1_scale_dev the scale is l1_scale * *l1_scale_dev, read on the device
    int l1;
    float l1_scale;
    const float* l1_scale_dev;
    // the inner units: strips [in_s0, in_s1) x segments [in_g0, in_g1), those
    // that run one staged row loop with plain stores (inv_inner_rect); a level
    // runs them in one kernel and every other unit in a second one
    int in_s0, in_s1, in_g0, in_g1;
    // adjoint: the units cover the quads and quad rows [-ext, n + ext) of the
    // extended domain (ext = 2; 0 for the inverse); outputs outside the image
    // go to `side` (adj_side_floats floats) for adj_fold_kernel
    int ext;
    // edge units (UNITS_EDGE) run in edge_split pieces of ceil(seg_rows /
    // edge_split) quad rows each: more, shorter row chains for the units that
    // run beside the inner ones
    int edge_split;
    float* side;
};

// The side buffer of one adjoint level of an h x w input: the four extended
// columns on each side of every row -4 .. h+3 (8 per row, corners included),
// then the four extended rows above and below, w columns each.
__host__ __device__ inline int64_t adj_side_floats(int h, int w) { return int64_t(8) * (h + 8) + int64_t(8) * w; }

// Persistent forward: one descriptor per (image, level), one entry per unit
// of work in queue order, counters of completed strips per (image, level,
// segment).  Offsets are in elements from the base pointers of PmlParams.
struct PmlDesc {
    int h, w, hq, wq, hh, wh;
    int n_strips, seg_rows;
    int src_is_ws;                 // level input: 0 the images, 1 the workspace
    int64_t src_off, src_pitch;    // compute-type elements
    int64_t coef_off, coef_pitch;  // coefficient elements (the image's origin)
    int ll_is_ct;                  // LL to the workspace (1) or the coefficients (0)
    int64_t ll_off, ll_pitch;
    int vec_lo, vec_hi, vec_ll;    // pair-store alignment for an aligned coefficient base
    int ctr_base;                  // first counter of this level's segments
    int dep_base, dep_need;        // previous level's counters (-1: none) and its strip count
};

struct PmlUnit {
    int desc, s, g;      // descriptor, strip, segment
    int dep_lo, dep_hi;  // segments of the previous level this unit reads
};

struct PmlParams {
    const void* in;
    void* coef;
    void* ws;
    const PmlDesc* descs;
    const PmlUnit* units;
    int n_units;
    unsigned* counters;
    unsigned* queue;
    int coef_vec;          // the coefficient base allows paired stores
    int test_drop_signal;  // test hook: queue entry 0 never signals completion
    unsigned* status;
    uint64_t timeout_ns;
};

// Grouped inverse / adjoint (plans of several images): one launch runs one
// level of up to INV_GROUP_MAX images, their parameters in one
// __grid_constant__ kernel parameter, as for the grouped forward.
constexpr int INV_GROUP_MAX = 160;
struct InvGroupImg {
    InvParams p;
    int u_begin[3];  // first unit of the image among the launch's units, per unit class
};
struct InvGroupLaunch {
    InvGroupImg img[INV_GROUP_MAX];
    int n_img;
    int n_units[3];  // per unit class
    int first;       // 1: the level's first group (its first launch is a plain launch)
};
static_assert(sizeof(InvGroupLaunch) <= 32764, "a grouped launch block fits the kernel parameter space");

// Unit classes of an inverse or adjoint level.  The inner units
// (inv_inner_rect) run one staged row loop with plain stores; the edge units
// (every other unit, each in inv_edge_split pieces of its segment) copy from
// mirrored (inverse) or zero-filled (adjoint) positions and the adjoint's route
// their stores.  A level runs the inner units in one launch and the edge units
// in a second, separately compiled one.  Measured on the 16 x 4096^2 adjoint:
// both row loops in one kernel (its warps running either) 1.6x slower at level
// 1, the edge loop for every unit 1.46x slower (128 registers against 96, and
// its per-lane predicates).  UNITS_ALL is every unit in segment-major order.
enum { UNITS_ALL = 0, UNITS_INNER = 1, UNITS_EDGE = 2 };
__host__ __device__ inline int inv_edge_split(const InvParams& p) { return p.edge_split > 1 ? p.edge_split : 1; }
// number of units of class cls (edge units counted in pieces)
__host__ __device__ inline int inv_class_units(const InvParams& p, int cls) {
    const int inner = (p.in_s1 - p.in_s0) * (p.in_g1 - p.in_g0);
    return cls == UNITS_ALL ? p.n_units : (cls == UNITS_INNER ? inner : (p.n_units - inner) * inv_edge_split(p));
}
// Strip s, segment g and (edge units) piece k of the lu-th unit of class cls;
// UNITS_ALL and UNITS_INNER in segment-major order.
__host__ __device__ inline void inv_class_unit(const InvParams& p, int cls, int lu, int& s, int& g, int& k) {
    k = 0;
    if (cls == UNITS_ALL) {
        s = lu % p.n_strips;
        g = lu / p.n_strips;
        return;
    }
    if (cls == UNITS_INNER) {
        const int ns = p.in_s1 - p.in_s0;
        s = p.in_s0 + lu % ns;
        g = p.in_g0 + lu / ns;
        return;
    }
    k = lu % inv_edge_split(p);
    lu /= inv_edge_split(p);
    if (p.in_s1 > p.in_s0 && p.in_g1 > p.in_g0) {
        // segments above the inner ones (whole rows of strips), then for each
        // inner segment its strips left and right of the inner ones, then the
        // segments below
        const int top = p.in_g0 * p.n_strips;
        if (lu < top) {
            s = lu % p.n_strips;
            g = lu / p.n_strips;
            return;
        }
        lu -= top;
        const int side = p.n_strips - (p.in_s1 - p.in_s0);
        const int mid = (p.in_g1 - p.in_g0) * side;
        if (lu < mid) {
            g = p.in_g0 + lu / side;
            const int j = lu % side;
            s = j < p.in_s0 ? j : p.in_s1 + (j - p.in_s0);
            return;
        }
        lu -= mid;
        s = lu % p.n_strips;
        g = p.in_g1 + lu / p.n_strips;
        return;
    }
    s = lu % p.n_strips;
    g = lu / p.n_strips;
}

int launch_inv_group_f32(int wav, int scheme, const InvGroupLaunch& g, int grid, int pdl, int cls, cudaStream_t s);
int launch_inv_group_f16(int wav, int scheme, const InvGroupLaunch& g, int grid, int pdl, int cls, cudaStream_t s);
int launch_inv_group_bf16(int wav, int scheme, const InvGroupLaunch& g, int grid, int pdl, int cls, cudaStream_t s);
int launch_inv_group_i32(int wav, int scheme, const InvGroupLaunch& g, int grid, int pdl, int cls, cudaStream_t s);
int launch_adj_group_f32(const InvGroupLaunch& g, int grid, int pdl, int cls, cudaStream_t s);
// the fold E^T of the adjoint levels in a grouped launch block / of one level
int launch_adj_fold_group(const InvGroupLaunch& g, int pdl, cudaStream_t s);
int launch_adj_fold(const InvParams& p, cudaStream_t s);

// Two forward levels in one launch (fused.cuh): level l comes through the
// tensor maps, level l+1 reads the level-l low-low band from a ring of rows in
// shared memory, so that band never reaches global memory.  A block owns `own`
// low-low columns (level l+1 input columns) and seg2 level l+1 quad rows; the
// last segment has at least two rows.
struct FusedParams {
    FwdParams l1, l2;  // l1.ll is not written
    int own, n_cols, seg2, n_segs, n_items;
    unsigned* status;
    uint64_t timeout_ns;
};
constexpr int FUSED_W1 = 9, FUSED_W2 = 5;           // producer (level l) and consumer (level l+1) warps
constexpr int FUSED_OWN_MAX = 60 * FUSED_W1 - 8;    // 4 halo columns each side
constexpr int FUSED_QR = 3, FUSED_NST = 3;          // producer stage ring

int launch_fused_f32(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FusedParams& p,
                     int grid, cudaStream_t s);
int launch_fused_f16(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FusedParams& p,
                     int grid, cudaStream_t s);
int launch_fused_bf16(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FusedParams& p,
                      int grid, cudaStream_t s);
int launch_fused_i32(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FusedParams& p,
                     int grid, cudaStream_t s);
int fused_blocks_per_sm(int wav, int scheme, int coef_dtype);

// Grouped forward (plans of several images): one launch runs one level of up
// to GROUP_MAX images with the single-image kernel's row loop.  The images'
// tensor maps and parameters are one __grid_constant__ kernel parameter (read
// from the constant bank where used); unit u belongs to the image whose
// [u_begin, u_begin + n_units) holds it.
constexpr int GROUP_MAX = 76;
struct GroupImg {
    FwdParams p;
    int u_begin;
};
struct GroupLaunch {
    CUtensorMap maps[2 * GROUP_MAX];  // [2i] box, [2i+1] single row of image i
    GroupImg img[GROUP_MAX];
    int n_img, n_units;
    int wait_prev;  // 1: the first launch of a level (its inputs come from earlier launches)
};
static_assert(sizeof(GroupLaunch) <= 32764, "a grouped launch block fits the kernel parameter space");

// forward launch configuration
struct FwdCfg {
    int ql, qr, nst, nw;  // quads per lane, quad rows per stage, stages per warp, warps per block
    int spec;             // 1: interior strips run a specialised row loop (larger kernel)
};

// geometry of a strip: 64*ql pixels loaded, 32*ql - 4 quads output
// halo quads on each side of a strip per wavelet (2; 4 for DD 13/7) and the
// quads a forward strip outputs
inline int wav_halo(int wav) { return wav == WAV_DD137 ? 4 : 2; }
inline int fwd_out_quads(const FwdCfg& c, int wav) { return 32 * c.ql - 2 * wav_halo(wav); }
inline int fwd_strip_px(const FwdCfg& c) { return 64 * c.ql; }

// kernel launchers, one translation unit per coefficient type; they return a
// cudaError_t value
int launch_forward_f32(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p,
                       int grid, const FwdCfg& cfg, cudaStream_t s);
int launch_forward_f16(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p,
                       int grid, const FwdCfg& cfg, cudaStream_t s);
int launch_forward_bf16(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p,
                        int grid, const FwdCfg& cfg, cudaStream_t s);
int launch_forward_i32(int wav, int scheme, const CUtensorMap& box, const CUtensorMap& row, const FwdParams& p,
                       int grid, const FwdCfg& cfg, cudaStream_t s);
int launch_group_f32(int wav, int scheme, const GroupLaunch& g, int grid, const FwdCfg& cfg, int pdl, cudaStream_t s);
int launch_group_f16(int wav, int scheme, const GroupLaunch& g, int grid, const FwdCfg& cfg, int pdl, cudaStream_t s);
int launch_group_bf16(int wav, int scheme, const GroupLaunch& g, int grid, const FwdCfg& cfg, int pdl, cudaStream_t s);
int launch_group_i32(int wav, int scheme, const GroupLaunch& g, int grid, const FwdCfg& cfg, int pdl, cudaStream_t s);

int launch_inverse_f32(int wav, int scheme, const InvParams& p, int grid, int pdl, int cls, cudaStream_t s);
int launch_inverse_f16(int wav, int scheme, const InvParams& p, int grid, int pdl, int cls, cudaStream_t s);
int launch_inverse_bf16(int wav, int scheme, const InvParams& p, int grid, int pdl, int cls, cudaStream_t s);
int launch_inverse_i32(int wav, int scheme, const InvParams& p, int grid, int pdl, int cls, cudaStream_t s);
int launch_adjoint_f32(const InvParams& p, int grid, int pdl, int cls, cudaStream_t s);

// The persistent launch loads with TMA through a device-resident table of
// two tensor maps (a box and a single row) per (image, level) descriptor,
// written when the plan first runs on a set of buffers; use_tma = 0 selects
// the cp.async loader instead (DWT2_PML_CPASYNC, for tests).
struct PmlLaunch {
    const CUtensorMap* maps;  // device table: [2*desc] box, [2*desc+1] single row
    PmlParams base;
    int use_tma;
};

int launch_pml_f32(int wav, int scheme, const PmlLaunch& p, int grid, cudaStream_t s);
int launch_pml_f16(int wav, int scheme, const PmlLaunch& p, int grid, cudaStream_t s);
int launch_pml_bf16(int wav, int scheme, const PmlLaunch& p, int grid, cudaStream_t s);
int launch_pml_i32(int wav, int scheme, const PmlLaunch& p, int grid, cudaStream_t s);
int pml_blocks_per_sm(int wav, int scheme, int coef_dtype);

// resident blocks per SM of a forward / inverse launch (0 on error)
int forward_blocks_per_sm(int wav, int scheme, int coef_dtype, const FwdCfg& cfg);
int inverse_blocks_per_sm(int wav, int scheme, int coef_dtype, bool adjoint);  // the inner-unit kernel

// the forward configurations compiled in (index 0 is the default); one with
// no resident block (forward_blocks_per_sm 0) is skipped by the tuner
constexpr int N_FWD_CFGS = 5;
extern const FwdCfg FWD_CFGS[N_FWD_CFGS];
size_t fwd_smem_bytes_of(const FwdCfg& c);
// the persistent kernel's fixed configuration
constexpr int PML_QL = 2, PML_QR = 3, PML_NST = 3, PML_NW = 4;
constexpr int INV_NW = 4;
constexpr int INV_QL = 2;
constexpr int INV_QR = 3, INV_NST = 3;  // staged inverse / adjoint ring
constexpr int INV_OUT_Q = 32 * INV_QL - 4;
inline int inv_out_quads(int wav) { return 32 * INV_QL - 2 * wav_halo(wav); }

}  // namespace dwt2

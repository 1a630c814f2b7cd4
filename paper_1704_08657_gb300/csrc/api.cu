// api.cu -- the C ABI of libdwt2 (include/dwt2.h): plan validation,
// workspace layout, tensor-map encoding and the per-level launches.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/dwt2.h"
#include "internal.h"

using namespace dwt2;

namespace {

struct LevelGeom {
    int h, w, hq, wq, hh, wh;
};

LevelGeom level_geom(int h, int w) {
    LevelGeom g;
    g.h = h;
    g.w = w;
    g.hq = (h + 1) / 2;
    g.wq = (w + 1) / 2;
    g.hh = h / 2;
    g.wh = w / 2;
    return g;
}

int64_t round4(int64_t v) { return (v + 3) / 4 * 4; }
size_t align256(size_t v) { return (v + 255) / 256 * 256; }

size_t dtype_size(int dt) { return (dt == DT_F16 || dt == DT_BF16) ? 2 : 4; }

struct ImagePlan {
    dwt2_image_desc d;
    std::vector<LevelGeom> lv;   // lv[l] = input geometry of level l (0-based)
    std::vector<size_t> ws_off;  // ws_off[l] = byte offset of level l's LL band (l < levels-1)
    std::vector<size_t> side_off;  // CDF 9/7: byte offset of level l's adjoint side buffer
};

// decomposition of one level into (strip, segment) units
struct Decomp {
    int n_strips, seg_rows, n_segs, n_units;
};

// Work decomposition of one level into units of seg_rows quad rows of one
// strip, dealt round-robin in segment-major order so that the warps at work
// at any moment cover one compact band of image rows (DRAM page and TLB
// locality; contiguous per-warp ranges that spread the warps over the whole
// image measured ~2x slower).  The segment height is chosen to minimise
// rounds x (rows + 4 rows of warm-up), where a round is one unit for every
// resident warp, over heights up to SEG_MAX so that the band stays small
// (heights of 32-56 rows measured best on 16384^2; 64-256 were 5-30 % slower).
// seg_override > 0 forces a height; balanced_env selects contiguous ranges.
constexpr int SEG_MIN = 8, SEG_MAX = 48, MIN_ROWS = 16;

Decomp decompose(const LevelGeom& g, int out_q, int sm_count, int blocks_per_sm, int nw, int seg_override,
                 int balanced_env, int* grid, int* balanced) {
    Decomp d;
    d.n_strips = (g.wq + out_q - 1) / out_q;
    const int64_t total = int64_t(g.hq) * d.n_strips;
    const int64_t max_warps = int64_t(sm_count) * std::max(blocks_per_sm, 1) * nw;
    if (balanced_env) {
        const int64_t warps = std::max<int64_t>(1, std::min(max_warps, (total + MIN_ROWS - 1) / MIN_ROWS));
        *grid = int((warps + nw - 1) / nw);
        *balanced = 1;
        d.seg_rows = g.hq;
        d.n_segs = 1;
        d.n_units = d.n_strips;
        return d;
    }
    int best = std::min(seg_override > 0 ? seg_override : SEG_MAX, g.hq);
    if (seg_override <= 0) {
        int64_t best_cost = INT64_MAX;
        for (int seg = std::min(SEG_MIN, g.hq); seg <= std::min(SEG_MAX, g.hq); ++seg) {
            const int64_t units = int64_t((g.hq + seg - 1) / seg) * d.n_strips;
            const int64_t rounds = (units + max_warps - 1) / max_warps;
            const int64_t cost = rounds * (seg + 4);
            if (cost < best_cost) best_cost = cost, best = seg;
        }
    }
    d.seg_rows = best;
    d.n_segs = (g.hq + d.seg_rows - 1) / d.seg_rows;
    d.n_units = d.n_segs * d.n_strips;
    *grid = (d.n_units + nw - 1) / nw;
    *balanced = 0;
    return d;
}

// driver entry point for TMA descriptors
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2-D map over a w x h array of 4-byte elements with row pitch `pitch`
// elements; box = box_w x box_rows.
int encode_map(CUtensorMap* m, const void* base, int w, int h, int64_t pitch, int box_w, int box_rows,
               bool is_int) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return DWT2_ERR_CUDA;
    cuuint64_t dims[2] = {cuuint64_t(w), cuuint64_t(h)};
    cuuint64_t strides[1] = {cuuint64_t(pitch) * 4};
    cuuint32_t box[2] = {cuuint32_t(box_w), cuuint32_t(box_rows)};
    cuuint32_t estr[2] = {1u, 1u};
    CUresult r = enc(m, is_int ? CU_TENSOR_MAP_DATA_TYPE_INT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                     const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? DWT2_OK : DWT2_ERR_MISALIGNED;
}

int env_int(const char* name, int dflt) {
    const char* v = getenv(name);
    return (v && *v) ? atoi(v) : dflt;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// The inverse and the adjoint do not depend on how the forward was scheduled:
// plans of the polyconvolution and convolution schemes run the non-separable
// lifting inverse and adjoint kernels.
int inv_scheme(int scheme) { return scheme > DWT2_SEP_LIFTING ? DWT2_NONSEP : scheme; }

}  // namespace

struct dwt2_plan_s {
    int wavelet, levels, in_dtype, coef_dtype, scheme, n_images;
    unsigned flags;
    std::vector<ImagePlan> imgs;
    size_t ws_bytes;
    size_t ws_levels;  // bytes the forward and the inverse use (the low-low bands)
    unsigned* d_status;
    int device, sm_count;
    int cfg_env, seg_env;           // DWT2_FWD_CFG, DWT2_SEG_ROWS
    int edge_split_env;             // DWT2_EDGE_SPLIT: pieces per inverse / adjoint edge unit
    int inv_edge_first;             // DWT2_INV_EDGE_FIRST: 1 / 0 edge units before / after a level's inner units, -1 adjoint first
    int cfg_bps[N_FWD_CFGS];        // resident blocks per SM of each forward configuration
    std::vector<int> lvl_cand;      // per level: tuning candidate, or -1 for cfg_env / seg_env
    int inv_bps;                    // resident blocks per SM of the inverse kernel
    int pdl;                        // per-level forward launches as programmatic dependents (DWT2_PDL)
    int overlap;                    // single image: inter-level overlap by segment counters (DWT2_LEVEL_OVERLAP)
    unsigned* d_lvl_ctr;            // the segment counters
    size_t n_lvl_ctr;
    int balanced_env;
    // fused level pairs: segment height in level l+1 quad rows (0: off) and
    // how many pairs, from level 0 on, may run fused
    int fuse_seg, fuse_pairs, fused_bps;
    uint64_t timeout_ns;
    // persistent forward: descriptors, queue-ordered units, counters + queue word
    bool persistent;
    int pml_bps, pml_seg, pml_force_cpasync, pml_lag_pct;
    std::vector<PmlDesc> h_descs;  // host copy (TMA maps are encoded per call from it)
    // grouped forward (several images, not persistent): the launch blocks of
    // every level (up to GROUP_MAX images each), built for one set of buffers
    // and one configuration and reused while those stay the same
    struct GroupCache {
        const void* in = nullptr;
        void* coef = nullptr;
        void* ws = nullptr;
        std::vector<int> cand;
        int cfg_env = -1, seg_env = -1, pdl = -1;
        std::vector<std::unique_ptr<GroupLaunch>> blocks;
        std::vector<int> level, grid, ci;  // per block
    } gcache;
    bool grouped;
    // grouped inverse / adjoint launch blocks (plans of several images), built
    // for one set of buffers and reused while those stay the same
    struct InvGroupCache {
        const void* coef = nullptr;
        void* out = nullptr;
        void* ws = nullptr;
        int adj = -1;
        std::vector<std::unique_ptr<InvGroupLaunch>> blocks;
        std::vector<int> level, grid, grid_edge;  // per block: the first launch's grid, the edge launch's
    } icache;
    PmlDesc* d_descs;
    PmlUnit* d_units;
    unsigned* d_counters;  // n_counters segment counters followed by the queue word
    int n_units, n_counters;
    // the persistent launch's tensor maps (two per descriptor) in device
    // memory, encoded for the input and workspace buffers they were last
    // written for
    CUtensorMap* d_maps;
    const void* maps_in;
    const void* maps_ws;
    // profiling: a ring of PROF_RING calls, one event pair per level each
    std::vector<cudaEvent_t> ev0, ev1;  // [slot * levels + level]
    bool prof_on;
    int prof_calls;  // calls recorded since profiling was enabled
};

namespace {
constexpr int PROF_RING = 256;
void prof_mark(dwt2_plan_t p, int level, bool start, cudaStream_t s) {
    if (!p->prof_on) return;
    const int slot = p->prof_calls % PROF_RING;
    cudaEventRecord(start ? p->ev0[slot * p->levels + level] : p->ev1[slot * p->levels + level], s);
}
}  // namespace

namespace {

// Queue order of the persistent forward.  Units of level 0 keep their natural
// order (image, segment, strip); a unit of level l gets the latest position of
// the level l-1 units it reads plus `lag`, about one GPU round of units, so
// that its inputs are normally complete when it is dequeued.
constexpr int PML_SEG_DEFAULT = 32;

int build_persistent(dwt2_plan_t p) {
    const int bps = pml_blocks_per_sm(p->wavelet, p->scheme, p->coef_dtype);
    if (bps <= 0) return DWT2_ERR_CUDA;
    p->pml_bps = bps;
    const int64_t lag = int64_t(p->sm_count) * bps * PML_NW * std::max(10, p->pml_lag_pct) / 100;
    const int L = p->levels;
    const size_t csz = dtype_size(p->coef_dtype);
    std::vector<PmlDesc> descs;
    std::vector<PmlUnit> units;
    std::vector<int64_t> keys;
    std::vector<int> levels_of;
    int ctr = 0;
    for (size_t i = 0; i < p->imgs.size(); ++i) {
        const ImagePlan& ip = p->imgs[i];
        std::vector<int64_t> seg_key_prev;  // latest key of each segment of level l-1
        int prev_base = -1, prev_need = 0, prev_seg = 1;
        for (int l = 0; l < L; ++l) {
            const LevelGeom& g = ip.lv[l];
            PmlDesc d;
            d.h = g.h, d.w = g.w, d.hq = g.hq, d.wq = g.wq, d.hh = g.hh, d.wh = g.wh;
            d.n_strips = (g.wq + fwd_out_quads(FwdCfg{PML_QL, PML_QR, PML_NST, PML_NW, 0}, p->wavelet) - 1) /
                         fwd_out_quads(FwdCfg{PML_QL, PML_QR, PML_NST, PML_NW, 0}, p->wavelet);
            d.seg_rows = std::min(p->pml_seg, g.hq);
            const int n_segs = (g.hq + d.seg_rows - 1) / d.seg_rows;
            d.src_is_ws = l > 0;
            d.src_off = (l == 0) ? ip.d.offset_elems : int64_t(ip.ws_off[l - 1] / 4);
            d.src_pitch = (l == 0) ? ip.d.pitch_elems : round4(ip.lv[l - 1].wq);
            d.coef_off = ip.d.offset_elems;
            d.coef_pitch = ip.d.pitch_elems;
            const bool last = (l == L - 1);
            d.ll_is_ct = !last;
            d.ll_off = last ? ip.d.offset_elems : int64_t(ip.ws_off[l] / 4);
            d.ll_pitch = last ? ip.d.pitch_elems : round4(g.wq);
            const bool cvec = (ip.d.pitch_elems % 2 == 0) && ((ip.d.offset_elems * csz) % (2 * csz) == 0);
            d.vec_lo = cvec;
            d.vec_hi = cvec && (g.wq % 2 == 0);
            d.vec_ll = last ? cvec : 1;
            d.ctr_base = ctr;
            d.dep_base = prev_base;
            d.dep_need = prev_need;
            const int di = int(descs.size());
            descs.push_back(d);
            std::vector<int64_t> seg_key(n_segs, 0);
            for (int gseg = 0; gseg < n_segs; ++gseg) {
                const int R0 = gseg * d.seg_rows, R1 = std::min(R0 + d.seg_rows, g.hq);
                int dlo = 0, dhi = -1;
                int64_t key = int64_t(keys.size());
                if (l > 0) {
                    // input rows this unit can touch (warm-up, pipeline lag, stage
                    // rounding, mirrored rows), as rows of the level l-1 low-low band
                    int lo = std::max(0, 2 * R0 - 4);
                    const int hi = std::min(g.h, 2 * R1 + 8);
                    if (2 * R1 + 8 > g.h) lo = std::max(0, std::min(lo, g.h - 9));
                    dlo = lo / prev_seg;
                    dhi = (hi - 1) / prev_seg;
                    int64_t kmax = 0;
                    for (int q = dlo; q <= dhi; ++q) kmax = std::max(kmax, seg_key_prev[q]);
                    key = kmax + lag;
                }
                for (int s = 0; s < d.n_strips; ++s) {
                    units.push_back(PmlUnit{di, s, gseg, dlo, dhi});
                    keys.push_back(l == 0 ? int64_t(keys.size()) : key);
                    levels_of.push_back(l);
                }
                seg_key[gseg] = keys.back();
            }
            seg_key_prev.swap(seg_key);
            prev_base = ctr;
            prev_need = d.n_strips;
            prev_seg = d.seg_rows;
            ctr += n_segs;
        }
    }
    // stable sort by key (ties: lower level first)
    std::vector<int> order(units.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = int(i);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (keys[a] != keys[b]) return keys[a] < keys[b];
        return levels_of[a] < levels_of[b];
    });
    std::vector<PmlUnit> sorted(units.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = units[order[i]];
    p->n_units = int(sorted.size());
    p->n_counters = ctr;
    p->h_descs = descs;
    if (p->d_descs) cudaFree(p->d_descs);
    if (p->d_units) cudaFree(p->d_units);
    if (p->d_counters) cudaFree(p->d_counters);
    if (p->d_maps) cudaFree(p->d_maps);
    p->d_descs = nullptr;
    p->d_units = nullptr;
    p->d_counters = nullptr;
    p->d_maps = nullptr;
    p->maps_in = p->maps_ws = nullptr;
    if (cudaMalloc(&p->d_maps, 2 * descs.size() * sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMalloc(&p->d_descs, descs.size() * sizeof(PmlDesc)) != cudaSuccess ||
        cudaMalloc(&p->d_units, sorted.size() * sizeof(PmlUnit)) != cudaSuccess ||
        cudaMalloc(&p->d_counters, (size_t(ctr) + 1) * sizeof(unsigned)) != cudaSuccess ||
        cudaMemcpy(p->d_descs, descs.data(), descs.size() * sizeof(PmlDesc), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_units, sorted.data(), sorted.size() * sizeof(PmlUnit), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cudaGetLastError();
        return DWT2_ERR_CUDA;
    }
    return DWT2_OK;
}

// The parameters of one image's inverse (or adjoint) level, without the
// decomposition into units.
InvParams inv_level_params(dwt2_plan_t p, const ImagePlan& ip, int l, const void* coef, void* out, void* workspace,
                           size_t csz, bool adj, bool l1, float l1_scale, const float* l1_scale_dev = nullptr) {
    const char* coef_img = static_cast<const char*>(coef) + ip.d.offset_elems * csz;
    char* out_img = static_cast<char*>(out) + ip.d.offset_elems * 4;
    char* wsb = static_cast<char*>(workspace);
    const LevelGeom& g = ip.lv[l];
    InvParams ipm;
    memset(&ipm, 0, sizeof(ipm));
    ipm.h = g.h, ipm.w = g.w, ipm.hq = g.hq, ipm.wq = g.wq, ipm.hh = g.hh, ipm.wh = g.wh;
    ipm.coef = coef_img;
    ipm.coef_pitch = ip.d.pitch_elems;
    const bool coarsest = (l == p->levels - 1);
    if (coarsest) {
        ipm.ll = coef_img;
        ipm.ll_pitch = ip.d.pitch_elems;
        ipm.ll_is_ct = 0;
    } else {
        ipm.ll = wsb + ip.ws_off[l];
        ipm.ll_pitch = round4(g.wq);
        ipm.ll_is_ct = 1;
    }
    if (l == 0) {
        ipm.out = out_img;
        ipm.out_pitch = ip.d.pitch_elems;
    } else {
        ipm.out = wsb + ip.ws_off[l - 1];
        ipm.out_pitch = round4(g.w);  // = round4(wq of level l-1)
    }
    const bool cvec = (ip.d.pitch_elems % 2 == 0) && aligned(coef_img, 2 * csz);
    ipm.vec_in_lo = cvec;
    ipm.vec_in_hi = cvec && (g.wq % 2 == 0);
    ipm.vec_ll = coarsest ? cvec : 1;
    ipm.vec_out = (ipm.out_pitch % 4 == 0) && aligned(ipm.out, 16);
    ipm.status = p->d_status;
    ipm.timeout_ns = p->timeout_ns;
    ipm.l1 = l1;
    ipm.l1_scale = l1_scale;
    ipm.l1_scale_dev = l1_scale_dev;
    // the adjoint runs on the domain extended by two quads past every edge
    ipm.ext = adj ? 2 : 0;
    ipm.side = adj ? reinterpret_cast<float*>(wsb + ip.side_off[l]) : nullptr;
    return ipm;
}

// The inner units of one inverse / adjoint level, in_s0 .. in_g1 of q: the
// units whose band rows all take paired staged copies (pair-aligned bands)
// from inside the band columns (the strip's first pixel >= 0 and its quads
// within the odd-column band) and, for the adjoint, whose output rows all lie
// inside the image (none of its outputs is an extended position).  Each
// condition is monotone in the strip or the segment index, so these units
// form a rectangle; the kernels run them with one staged row loop and plain
// stores, and every other unit in a second launch.
void inv_inner_rect(InvParams& q, int wavelet, bool adj) {
    const int hq_ = wav_halo(wavelet), outq = 64 - 2 * hq_;
    const bool staged = q.vec_in_lo && q.vec_in_hi && q.vec_ll;
    int s0 = q.n_strips, s1 = 0, g0 = q.n_segs, g1 = 0;
    for (int st = 0; st < q.n_strips && staged; ++st) {
        const int x0 = st * (2 * outq) - 2 * hq_ - 2 * q.ext;
        const bool in = (x0 >= 0) && (x0 / 2 + 64 <= q.wh);
        if (in) s0 = std::min(s0, st), s1 = st + 1;
    }
    for (int g = 0; g < q.n_segs; ++g) {
        const int R0 = g * q.seg_rows - q.ext, R1 = std::min(R0 + q.seg_rows, q.hq + q.ext);
        // adjoint: no output row outside the image (R1 <= hh: every odd pixel row exists)
        const bool in = !adj || ((R0 >= 0) && (R1 <= q.hh));
        if (in) g0 = std::min(g0, g), g1 = g + 1;
    }
    // the strip and the segment ranges are kept apart (an adjoint level uses
    // the inner strips also when it has no inner segment)
    if (s0 >= s1) s0 = s1 = 0;
    if (g0 >= g1) g0 = g1 = 0;
    q.in_s0 = s0, q.in_s1 = s1, q.in_g0 = g0, q.in_g1 = g1;
}

// Plans of several images: every level, coarsest first, as launches of up to
// INV_GROUP_MAX images.  The segment height of a launch is the one of
// INV_SEG_MIN .. INV_SEG_MAX quad rows that minimises rounds x (rows + the
// pipeline's WARM + LAG = 4 rows), a round being one unit for every resident
// warp: the whole level when it fits one round (the coarse levels, whose
// time is one unit's row chain), 32-row segments on the large ones.
constexpr int INV_SEG_MIN = 8, INV_SEG_MAX = 32;

// Edge units run in two pieces of a 16-32-row segment when twice their number
// still fits one round of resident warps: they are then a latency-bound row
// chain, which a piece halves for four more warm-up rows; when they fill more
// than a round the extra rows cost more than the shorter chains save
// (measured on the 16 x 4096^2 adjoint: level 3 35 -> 25 us, level 2 37 ->
// 45 us with pieces).
int inv_edge_pieces(int seg, int64_t edge_units, int64_t max_warps, int env) {
    if (env > 0) return env;
    return seg >= 16 && 2 * edge_units <= max_warps ? 2 : 1;
}

int inv_group_seg(const std::vector<InvParams>& ps, int64_t max_warps, int seg_env) {
    if (seg_env > 0) return seg_env;
    int best = INV_SEG_MAX;
    int64_t best_cost = INT64_MAX;
    for (int seg = INV_SEG_MAX; seg >= INV_SEG_MIN; --seg) {
        int64_t units = 0;
        for (const InvParams& q : ps) units += int64_t(q.n_strips) * ((q.hq + 2 * q.ext + seg - 1) / seg);
        const int64_t cost = (units + max_warps - 1) / max_warps * (seg + 4);
        if (cost < best_cost) best_cost = cost, best = seg;
    }
    return best;
}

// Launch order of a level's two unit classes (measured, not derived): the
// adjoint's edge units (routed stores, zero-filled copies, ~10 % of a level's
// units at 4096^2) launched before its inner units made the 16 x 4096^2 L1
// adjoint 2 % faster; the inverse's were 2 % faster after them (16384^2,
// 5 levels).  The first launch is a plain launch, the second a programmatic
// dependent that starts once the first has placed all its blocks.
std::array<int, 2> inv_class_order(dwt2_plan_t p, bool adj) {
    const bool edge_first = p->inv_edge_first < 0 ? adj : p->inv_edge_first != 0;
    if (edge_first) return {UNITS_EDGE, UNITS_INNER};
    return {UNITS_INNER, UNITS_EDGE};
}

int inv_group_build(dwt2_plan_t p, const void* coef, void* out, void* workspace, bool adj) {
    auto& ic = p->icache;
    ic.blocks.clear();
    ic.level.clear();
    ic.grid.clear();
    ic.grid_edge.clear();
    const int n = int(p->imgs.size());
    const size_t csz = adj ? 4 : dtype_size(p->coef_dtype);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return int64_t(p->imgs[a].d.h) * p->imgs[a].d.w > int64_t(p->imgs[b].d.h) * p->imgs[b].d.w;
    });
    const int inv_bps = adj ? inverse_blocks_per_sm(p->wavelet, inv_scheme(p->scheme), p->coef_dtype, true) : p->inv_bps;
    const int64_t max_warps = int64_t(p->sm_count) * std::max(inv_bps, 1) * INV_NW;
    for (int l = p->levels - 1; l >= 0; --l) {
        for (int i0 = 0; i0 < n; i0 += INV_GROUP_MAX) {
            std::unique_ptr<InvGroupLaunch> g(new (std::nothrow) InvGroupLaunch());
            if (!g) return DWT2_ERR_INVALID_ARG;
            std::vector<InvParams> ps;
            for (int k = 0; k < INV_GROUP_MAX && i0 + k < n; ++k) {
                const ImagePlan& ip = p->imgs[order[i0 + k]];
                InvParams ipm = inv_level_params(p, ip, l, coef, out, workspace, csz, adj, false, 0.f);
                // units over the quads and quad rows [-ext, n + ext)
                const int qw = ipm.wq + 2 * ipm.ext;
                ipm.n_strips = (qw + inv_out_quads(p->wavelet) - 1) / inv_out_quads(p->wavelet);
                ps.push_back(ipm);
            }
            const int seg = inv_group_seg(ps, max_warps, p->seg_env);
            int units[3] = {0, 0, 0};
            for (size_t k = 0; k < ps.size(); ++k) {
                InvParams& ipm = ps[k];
                const int qh = ipm.hq + 2 * ipm.ext;
                ipm.seg_rows = std::min(seg, qh);
                ipm.n_segs = (qh + ipm.seg_rows - 1) / ipm.seg_rows;
                ipm.n_units = ipm.n_segs * ipm.n_strips;
                ipm.edge_split = 1;
                inv_inner_rect(ipm, p->wavelet, adj);
            }
            int64_t edge_units = 0;
            for (const InvParams& q : ps) edge_units += inv_class_units(q, UNITS_EDGE);
            const int split = inv_edge_pieces(seg, edge_units, max_warps, p->edge_split_env);
            for (size_t k = 0; k < ps.size(); ++k) {
                InvParams& ipm = ps[k];
                ipm.edge_split = split;
                g->img[k].p = ipm;
                for (int c = 0; c < 3; ++c) {
                    g->img[k].u_begin[c] = units[c];
                    units[c] += inv_class_units(ipm, c);
                }
                g->n_img = int(k) + 1;
            }
            for (int c = 0; c < 3; ++c) g->n_units[c] = units[c];
            g->first = (i0 == 0);
            ic.grid.push_back((units[UNITS_INNER] + INV_NW - 1) / INV_NW);
            ic.grid_edge.push_back((units[UNITS_EDGE] + INV_NW - 1) / INV_NW);
            ic.level.push_back(l);
            ic.blocks.push_back(std::move(g));
        }
    }
    ic.coef = coef, ic.out = out, ic.ws = workspace, ic.adj = adj;
    return DWT2_OK;
}

int inverse_grouped(dwt2_plan_t p, const void* coef, void* out, void* workspace, cudaStream_t s, bool adj, bool l1,
                    float l1_scale, const float* l1_scale_dev) {
    auto& ic = p->icache;
    if (ic.blocks.empty() || ic.coef != coef || ic.out != out || ic.ws != workspace || ic.adj != int(adj)) {
        const int rc = inv_group_build(p, coef, out, workspace, adj);
        if (rc != DWT2_OK) {
            ic.blocks.clear();
            return rc;
        }
    }
    for (size_t b = 0; b < ic.blocks.size(); ++b) {
        InvGroupLaunch& g = *ic.blocks[b];
        for (int k = 0; k < g.n_img; ++k) {
            g.img[k].p.l1 = l1;
            g.img[k].p.l1_scale = l1_scale;
            g.img[k].p.l1_scale_dev = l1_scale_dev;
        }
        const int l = ic.level[b];
        if (b == 0 || ic.level[b - 1] != l) prof_mark(p, l, true, s);
        // the two unit classes in inv_class_order; the level's first launch
        // is a plain launch, the others programmatic dependents
        // (inv_group_kernel)
        bool first = g.first != 0;
        for (int cls : inv_class_order(p, adj)) {
            const int grid = cls == UNITS_EDGE ? ic.grid_edge[b] : ic.grid[b];
            if (grid == 0) continue;
            const int pdl = first ? 0 : 1;
            first = false;
            int e;
            if (adj) {
                e = launch_adj_group_f32(g, grid, pdl, cls, s);
            } else {
                const int sc = inv_scheme(p->scheme);
                switch (p->coef_dtype) {
                    case DWT2_F32: e = launch_inv_group_f32(p->wavelet, sc, g, grid, pdl, cls, s); break;
                    case DWT2_F16: e = launch_inv_group_f16(p->wavelet, sc, g, grid, pdl, cls, s); break;
                    case DWT2_BF16: e = launch_inv_group_bf16(p->wavelet, sc, g, grid, pdl, cls, s); break;
                    default: e = launch_inv_group_i32(p->wavelet, sc, g, grid, pdl, cls, s); break;
                }
            }
            if (e != cudaSuccess) return DWT2_ERR_CUDA;
        }
        const bool level_done = b + 1 == ic.blocks.size() || ic.level[b + 1] != l;
        if (adj && level_done) {
            // the fold of every image of the level, once all its units are stored
            for (size_t f = b + 1; f-- > 0 && ic.level[f] == l;)
                if (launch_adj_fold_group(*ic.blocks[f], f == b ? 0 : 1, s) != cudaSuccess) return DWT2_ERR_CUDA;
        }
        if (level_done) prof_mark(p, l, false, s);
    }
    if (p->prof_on) ++p->prof_calls;
    return DWT2_OK;
}

int forward_persistent(dwt2_plan_t p, const void* in, void* coef, void* workspace, cudaStream_t s) {
    const size_t csz = dtype_size(p->coef_dtype);
    PmlLaunch launch{};
    PmlLaunch* lp = &launch;
    PmlParams& pp = lp->base;
    pp.in = in;
    pp.coef = coef;
    pp.ws = workspace;
    pp.descs = p->d_descs;
    pp.units = p->d_units;
    pp.n_units = p->n_units;
    pp.counters = p->d_counters;
    pp.queue = p->d_counters + p->n_counters;
    pp.coef_vec = aligned(coef, 2 * csz);
    pp.test_drop_signal = (p->flags & DWT2_TESTONLY_DROP_SIGNAL) != 0;
    pp.status = p->d_status;
    pp.timeout_ns = p->timeout_ns;
    lp->use_tma = !p->pml_force_cpasync;
    lp->maps = p->d_maps;
    if (lp->use_tma && (p->maps_in != in || p->maps_ws != workspace)) {
        // (re)write the tensor maps for these buffers: outside any stream
        // capture, after the launches still reading the old ones
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return DWT2_ERR_CUDA;
        if (cs != cudaStreamCaptureStatusNone) return DWT2_ERR_INVALID_ARG;
        const bool is_int = p->wavelet == DWT2_CDF53_INT;
        const int bw = 64 * PML_QL;
        std::vector<CUtensorMap> maps(2 * p->h_descs.size());
        for (size_t i = 0; i < p->h_descs.size(); ++i) {
            const PmlDesc& d = p->h_descs[i];
            const char* base = d.src_is_ws ? static_cast<const char*>(workspace) : static_cast<const char*>(in);
            const void* src = base + d.src_off * 4;
            int rc = encode_map(&maps[2 * i], src, d.w, d.h, d.src_pitch, bw, 2 * PML_QR, is_int);
            if (rc == DWT2_OK) rc = encode_map(&maps[2 * i + 1], src, d.w, d.h, d.src_pitch, bw, 1, is_int);
            if (rc != DWT2_OK) return rc;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess ||
            cudaMemcpy(p->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice) !=
                cudaSuccess) {
            cudaGetLastError();
            return DWT2_ERR_CUDA;
        }
        p->maps_in = in;
        p->maps_ws = workspace;
    }
    if (cudaMemsetAsync(p->d_counters, 0, (size_t(p->n_counters) + 1) * sizeof(unsigned), s) != cudaSuccess)
        return DWT2_ERR_CUDA;
    const int grid = p->sm_count * p->pml_bps;
    prof_mark(p, 0, true, s);
    int e;
    switch (p->coef_dtype) {
        case DWT2_F32: e = launch_pml_f32(p->wavelet, p->scheme, launch, grid, s); break;
        case DWT2_F16: e = launch_pml_f16(p->wavelet, p->scheme, launch, grid, s); break;
        case DWT2_BF16: e = launch_pml_bf16(p->wavelet, p->scheme, launch, grid, s); break;
        default: e = launch_pml_i32(p->wavelet, p->scheme, launch, grid, s); break;
    }
    // the whole pyramid is one launch: it is timed as level 0; the other levels read 0
    prof_mark(p, 0, false, s);
    for (int l = 1; l < p->levels; ++l) {
        prof_mark(p, l, true, s);
        prof_mark(p, l, false, s);
    }
    if (p->prof_on) ++p->prof_calls;
    return e == cudaSuccess ? DWT2_OK : DWT2_ERR_CUDA;
}

// The output fields of one forward level of one image (geometry, band
// pointers, pair-store alignment); the work decomposition is left to the caller.
FwdParams level_outputs(dwt2_plan_t p, const ImagePlan& ip, int l, void* coef, void* workspace) {
    const size_t csz = dtype_size(p->coef_dtype);
    char* coef_img = static_cast<char*>(coef) + ip.d.offset_elems * csz;
    char* wsb = static_cast<char*>(workspace);
    const LevelGeom& g = ip.lv[l];
    FwdParams fp{};  // every field not set below (overlap, test hook) is zero
    fp.h = g.h, fp.w = g.w, fp.hq = g.hq, fp.wq = g.wq, fp.hh = g.hh, fp.wh = g.wh;
    fp.coef = coef_img;
    fp.coef_pitch = ip.d.pitch_elems;
    const bool last = (l == p->levels - 1);
    if (last) {
        fp.ll = coef_img;
        fp.ll_pitch = ip.d.pitch_elems;
        fp.ll_is_ct = 0;
    } else {
        fp.ll = wsb + ip.ws_off[l];
        fp.ll_pitch = round4(g.wq);
        fp.ll_is_ct = 1;
    }
    const bool coef_vec = (ip.d.pitch_elems % 2 == 0) && aligned(coef_img, 2 * csz);
    fp.vec_lo = coef_vec;
    fp.vec_hi = coef_vec && (g.wq % 2 == 0);
    fp.vec_ll = last ? coef_vec : 1;
    fp.status = p->d_status;
    fp.timeout_ns = p->timeout_ns;
    return fp;
}

// tensor maps over the input of level l of one image: a box of 2*qr rows and
// a single row, both 64*ql pixels wide
int level_maps(dwt2_plan_t p, const ImagePlan& ip, int l, const void* in, void* workspace, int ql, int qr,
               CUtensorMap* box, CUtensorMap* row) {
    const LevelGeom& g = ip.lv[l];
    const void* src = (l == 0) ? static_cast<const void*>(static_cast<const char*>(in) + ip.d.offset_elems * 4)
                               : static_cast<const void*>(static_cast<const char*>(workspace) + ip.ws_off[l - 1]);
    const int64_t src_pitch = (l == 0) ? ip.d.pitch_elems : round4(ip.lv[l - 1].wq);
    const bool is_int = p->wavelet == DWT2_CDF53_INT;
    int rc = encode_map(box, src, g.w, g.h, src_pitch, 64 * ql, 2 * qr, is_int);
    if (rc == DWT2_OK) rc = encode_map(row, src, g.w, g.h, src_pitch, 64 * ql, 1, is_int);
    return rc;
}

// Tuning candidates of one per-level forward launch: every compiled kernel
// configuration with the automatic segment height and a few fixed heights.
const int TUNE_SEGS[] = {0, 2, 4, 8, 12, 16, 24, 32};
constexpr int N_TUNE_SEGS = int(sizeof(TUNE_SEGS) / sizeof(TUNE_SEGS[0]));
constexpr int N_LVL_CANDS = N_FWD_CFGS * N_TUNE_SEGS;
constexpr int TUNE_BITS = 6, TUNE_LEVELS = 5;  // a plan's choice: 6 bits per level, levels >= 4 share one
static_assert(N_LVL_CANDS <= (1 << TUNE_BITS), "candidates fit the choice field");

// The launch configuration of one forward level of one image.
struct LevelLaunch {
    int ci;  // index into FWD_CFGS
    Decomp dc;
    int grid, balanced;
};

LevelLaunch level_launch(dwt2_plan_t p, const ImagePlan& ip, int l) {
    LevelLaunch ll;
    ll.ci = p->cfg_env;
    int seg = p->seg_env;
    const int cand = p->lvl_cand[l];
    if (cand >= 0) {
        ll.ci = cand / N_TUNE_SEGS;
        seg = TUNE_SEGS[cand % N_TUNE_SEGS];
    }
    const FwdCfg& cfg = FWD_CFGS[ll.ci];
    ll.dc = decompose(ip.lv[l], fwd_out_quads(cfg, p->wavelet), p->sm_count, p->cfg_bps[ll.ci], cfg.nw, seg, p->balanced_env,
                      &ll.grid, &ll.balanced);
    return ll;
}

// One forward level of one image.  dep_ctr / out_ctr: inter-level overlap
// (the FwdParams fields of those names); null for a launch that waits for the
// previous grid.
int forward_level(dwt2_plan_t p, const ImagePlan& ip, int l, const void* in, void* coef, void* workspace,
                  cudaStream_t s, const LevelLaunch& ll, const unsigned* dep_ctr = nullptr, int dep_need = 0,
                  int dep_seg = 1, unsigned* out_ctr = nullptr) {
    const FwdCfg& cfg = FWD_CFGS[ll.ci];
    CUtensorMap box, row;
    const int rc = level_maps(p, ip, l, in, workspace, cfg.ql, cfg.qr, &box, &row);
    if (rc != DWT2_OK) return rc;
    FwdParams fp = level_outputs(p, ip, l, coef, workspace);
    const Decomp& dc = ll.dc;
    fp.n_strips = dc.n_strips, fp.seg_rows = dc.seg_rows, fp.n_segs = dc.n_segs, fp.n_units = dc.n_units;
    fp.balanced = ll.balanced;
    fp.pdl = p->pdl;
    fp.dep_ctr = dep_ctr;
    fp.dep_need = dep_need;
    fp.dep_seg = dep_seg;
    fp.out_ctr = out_ctr;
    fp.test_drop = (p->flags & DWT2_TESTONLY_DROP_SIGNAL) != 0;
    int e;
    switch (p->coef_dtype) {
        case DWT2_F32: e = launch_forward_f32(p->wavelet, p->scheme, box, row, fp, ll.grid, cfg, s); break;
        case DWT2_F16: e = launch_forward_f16(p->wavelet, p->scheme, box, row, fp, ll.grid, cfg, s); break;
        case DWT2_BF16: e = launch_forward_bf16(p->wavelet, p->scheme, box, row, fp, ll.grid, cfg, s); break;
        default: e = launch_forward_i32(p->wavelet, p->scheme, box, row, fp, ll.grid, cfg, s); break;
    }
    return e == cudaSuccess ? DWT2_OK : DWT2_ERR_CUDA;
}

// Segment height of a grouped level when the tuner left it automatic: the
// units of many images fill the GPU, so no short segments are needed.
constexpr int GROUP_SEG_DEFAULT = 24;

// (Re)build the launch blocks of a grouped plan for these buffers.
int group_build(dwt2_plan_t p, const void* in, void* coef, void* workspace) {
    auto& gc = p->gcache;
    gc.blocks.clear();
    gc.level.clear();
    gc.grid.clear();
    gc.ci.clear();
    const int n = int(p->imgs.size());
    // groups are formed largest image first, so that the last launches of a
    // level (whose tails nothing overlaps) hold the smallest units
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return int64_t(p->imgs[a].d.h) * p->imgs[a].d.w > int64_t(p->imgs[b].d.h) * p->imgs[b].d.w;
    });
    for (int l = 0; l < p->levels; ++l) {
        int ci = p->cfg_env, seg = p->seg_env;
        if (p->lvl_cand[l] >= 0) {
            ci = p->lvl_cand[l] / N_TUNE_SEGS;
            seg = TUNE_SEGS[p->lvl_cand[l] % N_TUNE_SEGS];
        }
        if (seg <= 0) seg = GROUP_SEG_DEFAULT;
        const FwdCfg& cfg = FWD_CFGS[ci];
        const int outq = fwd_out_quads(cfg, p->wavelet);
        for (int i0 = 0; i0 < n; i0 += GROUP_MAX) {
            std::unique_ptr<GroupLaunch> g(new (std::nothrow) GroupLaunch());
            if (!g) return DWT2_ERR_INVALID_ARG;
            int units = 0;
            for (int k = 0; k < GROUP_MAX && i0 + k < n; ++k) {
                const ImagePlan& ip = p->imgs[order[i0 + k]];
                const int rc = level_maps(p, ip, l, in, workspace, cfg.ql, cfg.qr, &g->maps[2 * k], &g->maps[2 * k + 1]);
                if (rc != DWT2_OK) return rc;
                FwdParams fp = level_outputs(p, ip, l, coef, workspace);
                const LevelGeom& lg = ip.lv[l];
                fp.n_strips = (lg.wq + outq - 1) / outq;
                fp.seg_rows = std::min(seg, lg.hq);
                fp.n_segs = (lg.hq + fp.seg_rows - 1) / fp.seg_rows;
                fp.n_units = fp.n_segs * fp.n_strips;
                fp.balanced = 0;
                fp.pdl = p->pdl;
                g->img[k].p = fp;
                g->img[k].u_begin = units;
                units += fp.n_units;
                g->n_img = k + 1;
            }
            g->n_units = units;
            g->wait_prev = (i0 == 0);
            gc.grid.push_back((units + cfg.nw - 1) / cfg.nw);
            gc.level.push_back(l);
            gc.ci.push_back(ci);
            gc.blocks.push_back(std::move(g));
        }
    }
    gc.in = in, gc.coef = coef, gc.ws = workspace;
    gc.cand = p->lvl_cand;
    gc.cfg_env = p->cfg_env, gc.seg_env = p->seg_env, gc.pdl = p->pdl;
    return DWT2_OK;
}

// Plans of several images: every level as launches of up to GROUP_MAX images
// (programmatic dependents of one another), from the cached launch blocks.
int forward_grouped(dwt2_plan_t p, const void* in, void* coef, void* workspace, cudaStream_t s) {
    auto& gc = p->gcache;
    if (gc.blocks.empty() || gc.in != in || gc.coef != coef || gc.ws != workspace || gc.cand != p->lvl_cand ||
        gc.cfg_env != p->cfg_env || gc.seg_env != p->seg_env || gc.pdl != p->pdl) {
        const int rc = group_build(p, in, coef, workspace);
        if (rc != DWT2_OK) {
            gc.blocks.clear();
            return rc;
        }
    }
    for (size_t b = 0; b < gc.blocks.size(); ++b) {
        const int l = gc.level[b];
        if (b == 0 || gc.level[b - 1] != l) prof_mark(p, l, true, s);
        // the first launch of a level waits for every earlier launch (plain
        // stream order); the others overlap the launch before them
        const int pdl = gc.blocks[b]->wait_prev ? (l == 0 && p->pdl) : 1;
        const FwdCfg& cfg = FWD_CFGS[gc.ci[b]];
        int e;
        switch (p->coef_dtype) {
            case DWT2_F32: e = launch_group_f32(p->wavelet, p->scheme, *gc.blocks[b], gc.grid[b], cfg, pdl, s); break;
            case DWT2_F16: e = launch_group_f16(p->wavelet, p->scheme, *gc.blocks[b], gc.grid[b], cfg, pdl, s); break;
            case DWT2_BF16: e = launch_group_bf16(p->wavelet, p->scheme, *gc.blocks[b], gc.grid[b], cfg, pdl, s); break;
            default: e = launch_group_i32(p->wavelet, p->scheme, *gc.blocks[b], gc.grid[b], cfg, pdl, s); break;
        }
        if (e != cudaSuccess) return DWT2_ERR_CUDA;
        if (b + 1 == gc.blocks.size() || gc.level[b + 1] != l) prof_mark(p, l, false, s);
    }
    if (p->prof_on) ++p->prof_calls;
    return DWT2_OK;
}

// Single-image pyramid with inter-level overlap: the segment counters of
// levels 0 .. L-2 are cleared, then every level after the first waits on
// its predecessor's counters instead of its grid.
int forward_overlapped(dwt2_plan_t p, const void* in, void* coef, void* workspace, cudaStream_t s) {
    const ImagePlan& ip = p->imgs[0];
    const int L = p->levels;
    std::vector<LevelLaunch> lls(L);
    std::vector<size_t> base(L, 0);
    size_t n = 0;
    for (int l = 0; l < L; ++l) {
        lls[l] = level_launch(p, ip, l);
        if (lls[l].balanced) return DWT2_ERR_INVALID_ARG;  // counters need whole segments
        base[l] = n;
        if (l + 1 < L) n += size_t(lls[l].dc.n_segs);
    }
    if (n > p->n_lvl_ctr) return DWT2_ERR_INVALID_ARG;
    if (n && cudaMemsetAsync(p->d_lvl_ctr, 0, n * sizeof(unsigned), s) != cudaSuccess) return DWT2_ERR_CUDA;
    for (int l = 0; l < L; ++l) {
        prof_mark(p, l, true, s);
        const unsigned* dep = l > 0 ? p->d_lvl_ctr + base[l - 1] : nullptr;
        unsigned* out = l + 1 < L ? p->d_lvl_ctr + base[l] : nullptr;
        const int rc = forward_level(p, ip, l, in, coef, workspace, s, lls[l], dep,
                                     l > 0 ? lls[l - 1].dc.n_strips : 0, l > 0 ? lls[l - 1].dc.seg_rows : 1, out);
        if (rc != DWT2_OK) return rc;
        prof_mark(p, l, false, s);
    }
    if (p->prof_on) ++p->prof_calls;
    return DWT2_OK;
}

// Levels l and l+1 in one launch need a level-l input of at least 64 x 64
// (mirror rows of the low-low band stay inside a block's ring).
bool fused_eligible(const LevelGeom& g) { return g.h >= 64 && g.w >= 64; }

int forward_fused(dwt2_plan_t p, const ImagePlan& ip, int l, const void* in, void* coef, void* workspace,
                  cudaStream_t s) {
    CUtensorMap box, row;
    const int rc = level_maps(p, ip, l, in, workspace, 2, FUSED_QR, &box, &row);
    if (rc != DWT2_OK) return rc;
    FusedParams fp;
    fp.l1 = level_outputs(p, ip, l, coef, workspace);
    fp.l1.ll = nullptr;  // the low-low band stays on chip
    fp.l2 = level_outputs(p, ip, l + 1, coef, workspace);
    const LevelGeom& g2 = ip.lv[l + 1];
    fp.n_cols = (g2.w + FUSED_OWN_MAX - 1) / FUSED_OWN_MAX;
    fp.own = int(round4((g2.w + fp.n_cols - 1) / fp.n_cols));
    fp.seg2 = std::max(2, std::min(p->fuse_seg, g2.hq));  // the ring protocol needs segments of >= 2 rows
    fp.n_segs = (g2.hq + fp.seg2 - 1) / fp.seg2;
    if (fp.n_segs > 1 && g2.hq - (fp.n_segs - 1) * fp.seg2 < 2) --fp.n_segs;  // no one-row last segment
    fp.n_items = fp.n_cols * fp.n_segs;
    fp.status = p->d_status;
    fp.timeout_ns = p->timeout_ns;
    const int grid = std::min(fp.n_items, p->sm_count * p->fused_bps);
    int e;
    switch (p->coef_dtype) {
        case DWT2_F32: e = launch_fused_f32(p->wavelet, p->scheme, box, row, fp, grid, s); break;
        case DWT2_F16: e = launch_fused_f16(p->wavelet, p->scheme, box, row, fp, grid, s); break;
        case DWT2_BF16: e = launch_fused_bf16(p->wavelet, p->scheme, box, row, fp, grid, s); break;
        default: e = launch_fused_i32(p->wavelet, p->scheme, box, row, fp, grid, s); break;
    }
    return e == cudaSuccess ? DWT2_OK : DWT2_ERR_CUDA;
}

}  // namespace

extern "C" {

int dwt2_checked(void) {
#ifdef DWT2_CHECKED
    return 1;
#else
    return 0;
#endif
}

const char* dwt2_strerror(int code) {
    switch (code) {
        case DWT2_OK: return "ok";
        case DWT2_ERR_INVALID_ARG: return "invalid argument";
        case DWT2_ERR_UNSUPPORTED: return "unsupported wavelet / dtype / scheme combination";
        case DWT2_ERR_LEVELS_TOO_DEEP: return "too many levels for the image size (a level input side would be < 2)";
        case DWT2_ERR_MISALIGNED: return "misaligned pointer, offset or pitch";
        case DWT2_ERR_CUDA: return "CUDA runtime error";
        case DWT2_ERR_TIMEOUT: return "a bounded device wait expired";
        case DWT2_ERR_DEVICE_CHECK: return "a device-side bounds check tripped";
        case DWT2_ERR_TOO_LARGE:
            return "image too large for dwt2_forward_noalloc (its static scratch holds 32 MiB of low-low bands)";
        default: return "unknown error";
    }
}

int dwt2_plan(dwt2_plan_t* out, int wavelet, int levels, int boundary, int in_dtype, int coef_dtype, int scheme,
              int n_images, const dwt2_image_desc* images, unsigned flags) {
    if (!out) return DWT2_ERR_INVALID_ARG;
    *out = nullptr;
    if (!images || n_images < 1 || levels < 1 || levels > 30) return DWT2_ERR_INVALID_ARG;
    if (boundary != DWT2_SYMMETRIC) return DWT2_ERR_INVALID_ARG;
    if (wavelet != DWT2_CDF97 && wavelet != DWT2_CDF53_INT && wavelet != DWT2_DD137) return DWT2_ERR_INVALID_ARG;
    if (scheme < DWT2_NONSEP || scheme > DWT2_NONSEP_CONV) return DWT2_ERR_INVALID_ARG;
    if (in_dtype < DWT2_F32 || in_dtype > DWT2_I32 || coef_dtype < DWT2_F32 || coef_dtype > DWT2_I32)
        return DWT2_ERR_INVALID_ARG;
    if (flags & ~(DWT2_FLAG_PERSISTENT | DWT2_TESTONLY_DROP_SIGNAL)) return DWT2_ERR_INVALID_ARG;
    if ((flags & DWT2_FLAG_PERSISTENT) && scheme > DWT2_SEP_LIFTING) return DWT2_ERR_UNSUPPORTED;
    if (wavelet == DWT2_CDF97) {
        if (in_dtype != DWT2_F32 || coef_dtype == DWT2_I32) return DWT2_ERR_UNSUPPORTED;
    } else if (wavelet == DWT2_DD137) {
        if (in_dtype != DWT2_F32 || coef_dtype == DWT2_I32) return DWT2_ERR_UNSUPPORTED;
        // the lifting schemes (no filter-bank form) and no persistent launch
        if (scheme != DWT2_NONSEP && scheme != DWT2_NONSEP_REDUCED && scheme != DWT2_SEP_LIFTING)
            return DWT2_ERR_UNSUPPORTED;
        if (flags & DWT2_FLAG_PERSISTENT) return DWT2_ERR_UNSUPPORTED;
    } else {
        if (in_dtype != DWT2_I32 || coef_dtype != DWT2_I32) return DWT2_ERR_UNSUPPORTED;
        if (scheme == DWT2_NONSEP_REDUCED) return DWT2_ERR_UNSUPPORTED;  // floor does not split
        // floor rounding belongs to the lifting steps: no filter-bank form
        if (scheme == DWT2_POLYCONV || scheme == DWT2_CONV || scheme == DWT2_NONSEP_CONV) return DWT2_ERR_UNSUPPORTED;
    }
    std::vector<ImagePlan> imgs(n_images);
    size_t ws = 0;
    for (int i = 0; i < n_images; ++i) {
        const dwt2_image_desc& d = images[i];
        if (d.h < 1 || d.w < 1 || d.pitch_elems < d.w || d.offset_elems < 0) return DWT2_ERR_INVALID_ARG;
        if (d.offset_elems % 4 != 0 || d.pitch_elems % 4 != 0) return DWT2_ERR_MISALIGNED;
        ImagePlan& ip = imgs[i];
        ip.d = d;
        int h = d.h, w = d.w;
        for (int l = 0; l < levels; ++l) {
            if (h < 2 || w < 2) return DWT2_ERR_LEVELS_TOO_DEEP;
            ip.lv.push_back(level_geom(h, w));
            h = (h + 1) / 2;
            w = (w + 1) / 2;
        }
        // the LL band of every level but the last has its own buffer, so that
        // levels may run concurrently (persistent launch)
        for (int l = 0; l + 1 < levels; ++l) {
            const LevelGeom& g = ip.lv[l];
            ip.ws_off.push_back(ws);
            ws += align256(size_t(g.hq) * size_t(round4(g.wq)) * 4);
        }
    }
    // the adjoint's side buffers (the outputs past the image edges of every
    // level, folded back after the level), after every low-low band
    size_t ws_levels = ws;
    if (wavelet == DWT2_CDF97) {
        for (ImagePlan& ip : imgs)
            for (int l = 0; l < levels; ++l) {
                ip.side_off.push_back(ws);
                ws += align256(size_t(adj_side_floats(ip.lv[l].h, ip.lv[l].w)) * 4);
            }
    }
    dwt2_plan_s* p = new (std::nothrow) dwt2_plan_s();
    if (!p) return DWT2_ERR_INVALID_ARG;
    p->wavelet = wavelet;
    p->levels = levels;
    p->in_dtype = in_dtype;
    p->coef_dtype = coef_dtype;
    p->scheme = scheme;
    p->n_images = n_images;
    p->flags = flags;
    p->imgs.swap(imgs);
    p->ws_bytes = ws;
    p->ws_levels = ws_levels;
    p->d_status = nullptr;
    p->prof_on = false;
    p->prof_calls = 0;
    p->timeout_ns = uint64_t(env_int("DWT2_TIMEOUT_MS", 2000)) * 1000000ull;
    p->seg_env = env_int("DWT2_SEG_ROWS", 0);
    p->edge_split_env = env_int("DWT2_EDGE_SPLIT", 0);
    p->inv_edge_first = std::max(-1, std::min(1, env_int("DWT2_INV_EDGE_FIRST", -1)));
    p->pdl = env_int("DWT2_PDL", 1) != 0;
    p->overlap = env_int("DWT2_LEVEL_OVERLAP", 1) != 0;
    p->d_lvl_ctr = nullptr;
    p->n_lvl_ctr = 0;
    p->lvl_cand.assign(levels, -1);
    p->fuse_seg = std::max(0, env_int("DWT2_FUSE_SEG", 0));
    p->fuse_pairs = std::max(0, env_int("DWT2_FUSE_PAIRS", 1));
    p->fused_bps = fused_blocks_per_sm(wavelet, scheme, coef_dtype);
    p->balanced_env = env_int("DWT2_BALANCED", 0);
    p->cfg_env = env_int("DWT2_FWD_CFG", 0);
    for (int c = 0; c < N_FWD_CFGS; ++c) p->cfg_bps[c] = forward_blocks_per_sm(wavelet, scheme, coef_dtype, FWD_CFGS[c]);
    // a configuration this plan's pipeline is not compiled for falls back to the default
    if (p->cfg_env < 0 || p->cfg_env >= N_FWD_CFGS || p->cfg_bps[p->cfg_env] <= 0) p->cfg_env = 0;
    p->inv_bps = inverse_blocks_per_sm(wavelet, inv_scheme(scheme), coef_dtype, false);
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess ||
        cudaMalloc(&p->d_status, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(p->d_status, 0, sizeof(unsigned)) != cudaSuccess) {
        if (p->d_status) cudaFree(p->d_status);
        delete p;
        cudaGetLastError();
        return DWT2_ERR_CUDA;
    }
    p->persistent = (flags & DWT2_FLAG_PERSISTENT) != 0;
    p->d_descs = nullptr;
    p->d_units = nullptr;
    p->d_counters = nullptr;
    p->d_maps = nullptr;
    p->maps_in = p->maps_ws = nullptr;
    p->n_units = p->n_counters = 0;
    p->pml_bps = 0;
    p->pml_seg = env_int("DWT2_PML_SEG_ROWS", PML_SEG_DEFAULT);
    p->pml_force_cpasync = env_int("DWT2_PML_CPASYNC", 0);
    p->pml_lag_pct = env_int("DWT2_PML_LAG_PCT", 300);
    if (p->pml_seg < 4) p->pml_seg = PML_SEG_DEFAULT;
    p->grouped = false;
    if (p->persistent) {
        const int rc = build_persistent(p);
        if (rc != DWT2_OK) {
            dwt2_destroy(p);
            return rc;
        }
    }
    if (n_images == 1 && !p->persistent && levels > 1) {
        // at most one segment per quad row and level
        size_t n = 0;
        for (int l = 0; l + 1 < levels; ++l) n += size_t(p->imgs[0].lv[l].hq);
        if (cudaMalloc(&p->d_lvl_ctr, n * sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            dwt2_destroy(p);
            return DWT2_ERR_CUDA;
        }
        p->n_lvl_ctr = n;
    }
    // several images: grouped launches of the single-image row loop
    if (n_images > 1) p->grouped = !p->persistent;
    *out = p;
    return DWT2_OK;
}

size_t dwt2_workspace_bytes(dwt2_plan_t p) { return p ? p->ws_bytes : 0; }

void dwt2_destroy(dwt2_plan_t p) {
    if (!p) return;
    if (p->d_status) cudaFree(p->d_status);
    if (p->d_descs) cudaFree(p->d_descs);
    if (p->d_units) cudaFree(p->d_units);
    if (p->d_counters) cudaFree(p->d_counters);
    if (p->d_maps) cudaFree(p->d_maps);
    if (p->d_lvl_ctr) cudaFree(p->d_lvl_ctr);
    for (cudaEvent_t e : p->ev0) cudaEventDestroy(e);
    for (cudaEvent_t e : p->ev1) cudaEventDestroy(e);
    delete p;
}

int dwt2_profile(dwt2_plan_t p, int enable) {
    if (!p) return DWT2_ERR_INVALID_ARG;
    if (enable && p->ev0.empty()) {
        const size_t n = size_t(PROF_RING) * p->levels;
        p->ev0.assign(n, nullptr);
        p->ev1.assign(n, nullptr);
        for (size_t i = 0; i < n; ++i) {
            if (cudaEventCreate(&p->ev0[i]) != cudaSuccess || cudaEventCreate(&p->ev1[i]) != cudaSuccess)
                return DWT2_ERR_CUDA;
        }
    }
    p->prof_on = enable != 0;
    p->prof_calls = 0;
    return DWT2_OK;
}

int dwt2_profile_read(dwt2_plan_t p, float* ms, int n) {
    if (!p || !ms || n < 0 || n > p->levels || p->ev0.empty() || p->prof_calls == 0) return DWT2_ERR_INVALID_ARG;
    const int calls = std::min(p->prof_calls, PROF_RING);
    for (int l = 0; l < n; ++l) {
        double sum = 0.0;
        for (int c = 0; c < calls; ++c) {
            const int slot = (p->prof_calls - 1 - c) % PROF_RING;
            float t = 0.f;
            if (cudaEventSynchronize(p->ev1[slot * p->levels + l]) != cudaSuccess ||
                cudaEventElapsedTime(&t, p->ev0[slot * p->levels + l], p->ev1[slot * p->levels + l]) != cudaSuccess)
                return DWT2_ERR_CUDA;
            sum += t;
        }
        ms[l] = float(sum / calls);
    }
    return DWT2_OK;
}

int dwt2_status(dwt2_plan_t p, void* stream) {
    if (!p) return DWT2_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned h = 0;
    if (cudaMemcpyAsync(&h, p->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaMemsetAsync(p->d_status, 0, sizeof(unsigned), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return DWT2_ERR_CUDA;
    if (h & DEV_TIMEOUT) return DWT2_ERR_TIMEOUT;
    if (h & DEV_CHECK) return DWT2_ERR_DEVICE_CHECK;
    return DWT2_OK;
}

int dwt2_forward(dwt2_plan_t p, const void* in, void* coef, void* workspace, void* stream) {
    if (!p || !in || !coef) return DWT2_ERR_INVALID_ARG;
    if (p->ws_levels && !workspace) return DWT2_ERR_INVALID_ARG;
    if (!aligned(in, 16) || (workspace && !aligned(workspace, 256))) return DWT2_ERR_MISALIGNED;
    const size_t csz = dtype_size(p->coef_dtype);
    if (!aligned(coef, csz)) return DWT2_ERR_MISALIGNED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->persistent) return forward_persistent(p, in, coef, workspace, s);
    if (p->grouped) return forward_grouped(p, in, coef, workspace, s);
    if (p->d_lvl_ctr && p->overlap && p->fuse_seg == 0 && !p->balanced_env)
        return forward_overlapped(p, in, coef, workspace, s);
    for (int l = 0; l < p->levels;) {
        bool fuse = p->fuse_seg > 0 && l / 2 < p->fuse_pairs && l % 2 == 0 && l + 1 < p->levels && p->fused_bps > 0;
        for (const ImagePlan& ip : p->imgs) fuse = fuse && fused_eligible(ip.lv[l]);
        prof_mark(p, l, true, s);
        for (const ImagePlan& ip : p->imgs) {
            const int rc = fuse ? forward_fused(p, ip, l, in, coef, workspace, s)
                                : forward_level(p, ip, l, in, coef, workspace, s, level_launch(p, ip, l));
            if (rc != DWT2_OK) return rc;
        }
        prof_mark(p, l, false, s);
        if (fuse) {  // the pair is one launch, timed as level l; level l+1 reads 0
            prof_mark(p, l + 1, true, s);
            prof_mark(p, l + 1, false, s);
        }
        l += fuse ? 2 : 1;
    }
    if (p->prof_on) ++p->prof_calls;
    return DWT2_OK;
}

// shared by the inverse and the adjoint: levels from the coarsest down.
// l1: adjoint of l1_scale * sum |detail coefficients| (coef holds coefficients).
static int run_inverse_like(dwt2_plan_t p, const void* coef, void* out, void* workspace, void* stream, bool adj,
                            bool l1 = false, float l1_scale = 0.f, const float* l1_scale_dev = nullptr) {
    if (!p || !coef || !out) return DWT2_ERR_INVALID_ARG;
    if ((adj ? p->ws_bytes : p->ws_levels) && !workspace) return DWT2_ERR_INVALID_ARG;
    if (workspace && !aligned(workspace, 256)) return DWT2_ERR_MISALIGNED;
    if (adj && p->wavelet != DWT2_CDF97) return DWT2_ERR_UNSUPPORTED;
    if (l1 && p->coef_dtype != DWT2_F32) return DWT2_ERR_UNSUPPORTED;
    const size_t csz = adj ? 4 : dtype_size(p->coef_dtype);
    if (!aligned(coef, csz) || !aligned(out, 4)) return DWT2_ERR_MISALIGNED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (l1_scale_dev && !aligned(l1_scale_dev, 4)) return DWT2_ERR_MISALIGNED;
    if (p->n_images > 1) return inverse_grouped(p, coef, out, workspace, s, adj, l1, l1_scale, l1_scale_dev);
    const int inv_bps = adj ? inverse_blocks_per_sm(p->wavelet, inv_scheme(p->scheme), p->coef_dtype, true) : p->inv_bps;
    for (int l = p->levels - 1; l >= 0; --l) {
        prof_mark(p, l, true, s);
        for (const ImagePlan& ip : p->imgs) {
            InvParams ipm = inv_level_params(p, ip, l, coef, out, workspace, csz, adj, l1, l1_scale, l1_scale_dev);
            int grid = 0, balanced = 0;
            LevelGeom ext_geom = ip.lv[l];  // units over the quads and quad rows [-ext, n + ext)
            ext_geom.wq += 2 * ipm.ext;
            ext_geom.hq += 2 * ipm.ext;
            const Decomp dc = decompose(ext_geom, inv_out_quads(p->wavelet), p->sm_count, inv_bps, INV_NW, p->seg_env,
                                        0, &grid, &balanced);
            ipm.n_strips = dc.n_strips, ipm.seg_rows = dc.seg_rows, ipm.n_segs = dc.n_segs, ipm.n_units = dc.n_units;
            ipm.balanced = 0;
            ipm.edge_split = 1;
            inv_inner_rect(ipm, p->wavelet, adj);
            ipm.edge_split = inv_edge_pieces(ipm.seg_rows, inv_class_units(ipm, UNITS_EDGE),
                                             int64_t(p->sm_count) * std::max(inv_bps, 1) * INV_NW, p->edge_split_env);
            // the two unit classes in inv_class_order, the second a
            // programmatic dependent of the first (no shared data)
            bool first = true;
            for (int cls : inv_class_order(p, adj)) {
                const int units = inv_class_units(ipm, cls);
                if (units == 0) continue;
                const int g = (units + INV_NW - 1) / INV_NW, pdl = first ? 0 : 1;
                first = false;
                int e;
                if (adj) {
                    e = launch_adjoint_f32(ipm, g, pdl, cls, s);
                } else {
                    const int sc = inv_scheme(p->scheme);
                    switch (p->coef_dtype) {
                        case DWT2_F32: e = launch_inverse_f32(p->wavelet, sc, ipm, g, pdl, cls, s); break;
                        case DWT2_F16: e = launch_inverse_f16(p->wavelet, sc, ipm, g, pdl, cls, s); break;
                        case DWT2_BF16: e = launch_inverse_bf16(p->wavelet, sc, ipm, g, pdl, cls, s); break;
                        default: e = launch_inverse_i32(p->wavelet, sc, ipm, g, pdl, cls, s); break;
                    }
                }
                if (e != cudaSuccess) return DWT2_ERR_CUDA;
            }
            // the adjoint: fold the outputs past the edges onto their mirrors
            if (adj && launch_adj_fold(ipm, s) != cudaSuccess) return DWT2_ERR_CUDA;
        }
        prof_mark(p, l, false, s);
    }
    if (p->prof_on) ++p->prof_calls;
    return DWT2_OK;
}

// Autotuning.  Per-level plans time every candidate of TUNE_SEGS x the
// compiled configurations on the whole pyramid, read each level's time from
// the plan's profile events and keep, level by level, the fastest candidate
// (the launches of different levels are independent).  The choice packs
// TUNE_BITS bits per level for the first TUNE_LEVELS levels; deeper levels use
// the last field.  Persistent plans try a few segment heights and queue lags.
static const int TUNE_PML_SEGS[] = {16, 24, 32, 48};
constexpr int N_TUNE_PML_SEGS = int(sizeof(TUNE_PML_SEGS) / sizeof(TUNE_PML_SEGS[0]));
// queue lag of the persistent order, in percent of one GPU round of units: a
// longer lag means fewer waits on counters and less L2 reuse of the low-low
// band (the 512-image batch measured 0.600 ms at 300, 0.577 at 500)
static const int TUNE_PML_LAGS[] = {300, 500, 800};
constexpr int N_TUNE_PML = N_TUNE_PML_SEGS * int(sizeof(TUNE_PML_LAGS) / sizeof(TUNE_PML_LAGS[0]));
// Fused level pairs are not among the candidates: on 16384^2 they measured
// 2.3x slower than the two per-level launches (the row pipeline is bound by
// instruction issue as much as by DRAM, and the fused kernel executes ~1.5x
// the instructions).  Plans enable them with DWT2_FUSE_SEG.

static int tune_fields(dwt2_plan_t p) { return std::min(p->levels, TUNE_LEVELS); }

// candidate c's configuration is compiled for this plan's pipeline
static bool cand_compiled(dwt2_plan_t p, int c) { return p->cfg_bps[c / N_TUNE_SEGS] > 0; }

// persistent plans tune one segment height for all levels
static bool tune_seg_only(dwt2_plan_t p) { return p->persistent; }

static int tune_apply(dwt2_plan_t p, int choice) {
    if (choice < 0) return DWT2_ERR_INVALID_ARG;
    if (tune_seg_only(p)) {
        if (choice >= N_TUNE_PML) return DWT2_ERR_INVALID_ARG;
        p->pml_seg = TUNE_PML_SEGS[choice % N_TUNE_PML_SEGS];
        p->pml_lag_pct = TUNE_PML_LAGS[choice / N_TUNE_PML_SEGS];
        return build_persistent(p);
    }
    const int nf = tune_fields(p);
    if (nf * TUNE_BITS < 31 && choice >= (1 << (nf * TUNE_BITS))) return DWT2_ERR_INVALID_ARG;
    for (int f = 0; f < nf; ++f) {
        const int c = (choice >> (f * TUNE_BITS)) & ((1 << TUNE_BITS) - 1);
        if (c >= N_LVL_CANDS || !cand_compiled(p, c)) return DWT2_ERR_INVALID_ARG;
    }
    for (int l = 0; l < p->levels; ++l) p->lvl_cand[l] = (choice >> (std::min(l, nf - 1) * TUNE_BITS)) & ((1 << TUNE_BITS) - 1);
    return DWT2_OK;
}

// Mean time of one whole forward call: the smallest of five means of eight
// calls, timed with one event pair around each group (no per-level events).
static int time_whole_call(dwt2_plan_t p, const void* in, void* coef, void* workspace, void* stream, float* ms) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return DWT2_ERR_CUDA;
    }
    int rc = DWT2_OK;
    for (int i = 0; i < 2 && rc == DWT2_OK; ++i) rc = dwt2_forward(p, in, coef, workspace, stream);
    for (int r = 0; r < 5 && rc == DWT2_OK; ++r) {
        cudaEventRecord(e0, s);
        for (int i = 0; i < 8 && rc == DWT2_OK; ++i) rc = dwt2_forward(p, in, coef, workspace, stream);
        cudaEventRecord(e1, s);
        float t = 0.f;
        if (rc == DWT2_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
            rc = DWT2_ERR_CUDA;
        if (rc == DWT2_OK) *ms = (r == 0) ? t / 8 : std::min(*ms, t / 8);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int dwt2_autotune(dwt2_plan_t p, const void* in, void* coef, void* workspace, void* stream, int* choice) {
    if (!p || !choice) return DWT2_ERR_INVALID_ARG;
    if (*choice >= 0) return tune_apply(p, *choice);
    const bool prof = p->prof_on;
    int rc = DWT2_OK;
    const int L = p->levels;
    const bool seg_only = tune_seg_only(p);
    // candidates are timed level by level with every level waiting for its
    // predecessor's grid (per-level events would misattribute overlapped levels)
    const int overlap = p->overlap;
    p->overlap = 0;
    const int n_cand = seg_only ? N_TUNE_PML : N_LVL_CANDS;
    std::vector<float> ms(size_t(n_cand) * L, 0.f);
    for (int c = 0; c < n_cand && rc == DWT2_OK; ++c) {
        if (seg_only) {
            rc = tune_apply(p, c);
        } else {
            if (!cand_compiled(p, c)) {  // never chosen
                for (int l = 0; l < L; ++l) ms[size_t(c) * L + l] = 1e30f;
                continue;
            }
            for (int l = 0; l < L; ++l) p->lvl_cand[l] = c;
        }
        for (int i = 0; i < 2 && rc == DWT2_OK; ++i) rc = dwt2_forward(p, in, coef, workspace, stream);
        // the smallest of three means of eight calls, per level
        float* mc = &ms[size_t(c) * L];
        for (int r = 0; r < 3 && rc == DWT2_OK; ++r) {
            std::vector<float> m(L, 0.f);
            rc = dwt2_profile(p, 1);
            for (int i = 0; i < 8 && rc == DWT2_OK; ++i) rc = dwt2_forward(p, in, coef, workspace, stream);
            if (rc == DWT2_OK) rc = dwt2_profile_read(p, m.data(), L);
            for (int l = 0; l < L && rc == DWT2_OK; ++l) mc[l] = (r == 0) ? m[l] : std::min(mc[l], m[l]);
        }
        p->prof_on = false;
    }
    p->prof_on = prof;
    p->prof_calls = 0;
    p->overlap = overlap;
    if (rc != DWT2_OK) return rc;
    int best = 0;
    if (seg_only) {
        // the whole call: a persistent launch is timed as level 0, the others read 0
        auto total = [&](int c) {
            float t = 0.f;
            for (int l = 0; l < L; ++l) t += ms[size_t(c) * L + l];
            return t;
        };
        for (int c = 1; c < n_cand; ++c)
            if (total(c) < total(best)) best = c;
    } else {
        const int nf = tune_fields(p);
        for (int f = 0; f < nf; ++f) {
            // the last field covers every deeper level: sum their times
            int bc = 0;
            float bt = 0.f;
            for (int c = 0; c < n_cand; ++c) {
                float t = 0.f;
                for (int l = f; l < (f == nf - 1 ? L : f + 1); ++l) t += ms[size_t(c) * L + l];
                if (c == 0 || t < bt) bc = c, bt = t;
            }
            best |= bc << (f * TUNE_BITS);
        }
        if ((overlap && p->d_lvl_ctr) || p->n_images > 1) {
            // With inter-level overlap (or the overlapping launches of the
            // image groups of a level) the fastest pyramid need not be made of
            // the fastest levels: time the per-level choice, the default, the
            // per-level choice on the first levels only and the best uniform
            // candidates (also with the first level's own fastest candidate)
            // and every configuration with automatic segment heights end to
            // end, overlap on, then refine the fastest field by field.
            std::vector<int> cands = {best, 0};
            // the per-level choice for the first k fields, the default after them
            for (int k = 1; k < nf; ++k) cands.push_back(best & ((1 << (k * TUNE_BITS)) - 1));
            std::vector<std::pair<float, int>> tot;
            for (int c = 0; c < n_cand; ++c) {
                float t = 0.f;
                for (int l = 0; l < L; ++l) t += ms[size_t(c) * L + l];
                tot.push_back({t, c});
            }
            std::sort(tot.begin(), tot.end());
            const int mask0 = (1 << TUNE_BITS) - 1;
            for (int k = 0; k < 3 && k < int(tot.size()); ++k) {
                int u = 0;
                for (int f = 0; f < nf; ++f) u |= tot[k].second << (f * TUNE_BITS);
                cands.push_back(u);
                // the same with the first level's own fastest candidate
                cands.push_back((u & ~mask0) | (best & mask0));
            }
            // every configuration with the automatic segment height on every level
            for (int ci = 0; ci < N_FWD_CFGS; ++ci) {
                if (!cand_compiled(p, ci * N_TUNE_SEGS)) continue;
                int u = 0;
                for (int f = 0; f < nf; ++f) u |= (ci * N_TUNE_SEGS) << (f * TUNE_BITS);
                cands.push_back(u);
            }
            std::sort(cands.begin(), cands.end());
            cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
            // interleaved rounds: every candidate is timed once per round and
            // keeps its best round, so that a drift of clocks or L2 contents
            // during tuning favours none of them
            std::vector<float> cand_ms(cands.size(), 0.f);
            for (int r = 0; r < 4 && rc == DWT2_OK; ++r) {
                for (size_t k = 0; k < cands.size() && rc == DWT2_OK; ++k) {
                    rc = tune_apply(p, cands[k]);
                    float t = 0.f;
                    if (rc == DWT2_OK) rc = time_whole_call(p, in, coef, workspace, stream, &t);
                    if (rc == DWT2_OK && (r == 0 || t < cand_ms[k])) cand_ms[k] = t;
                }
            }
            if (rc != DWT2_OK) return rc;
            size_t kb = 0;
            for (size_t k = 1; k < cands.size(); ++k)
                if (cand_ms[k] < cand_ms[kb]) kb = k;
            best = cands[kb];
            // Coordinate descent, end to end: each field in turn tries its
            // eight fastest per-level candidates and every configuration with
            // the automatic segment height, the others fixed; a change is kept
            // when the whole pyramid gets faster by more than 0.2 %.  A second
            // pass runs when the first changed anything.
            float cur = cand_ms[kb];
            bool changed = true;
            for (int pass = 0; pass < 2 && changed && rc == DWT2_OK; ++pass) {
                changed = false;
                for (int f = 0; f < nf && rc == DWT2_OK; ++f) {
                    const int l_end = (f == nf - 1) ? L : f + 1;
                    std::vector<std::pair<float, int>> lv;
                    for (int c = 0; c < n_cand; ++c) {
                        float t = 0.f;
                        for (int l = f; l < l_end; ++l) t += ms[size_t(c) * L + l];
                        if (t < 1e29f) lv.push_back({t, c});
                    }
                    std::sort(lv.begin(), lv.end());
                    std::vector<int> alts;
                    for (size_t k = 0; k < 8 && k < lv.size(); ++k) alts.push_back(lv[k].second);
                    for (int ci = 0; ci < N_FWD_CFGS; ++ci)
                        if (cand_compiled(p, ci * N_TUNE_SEGS)) alts.push_back(ci * N_TUNE_SEGS);
                    std::sort(alts.begin(), alts.end());
                    alts.erase(std::unique(alts.begin(), alts.end()), alts.end());
                    const int shift = f * TUNE_BITS;
                    for (int a : alts) {
                        if (((best >> shift) & mask0) == a) continue;
                        const int c = (best & ~(mask0 << shift)) | (a << shift);
                        float t = 0.f;
                        rc = tune_apply(p, c);
                        if (rc == DWT2_OK) rc = time_whole_call(p, in, coef, workspace, stream, &t);
                        if (rc != DWT2_OK) break;
                        if (t < cur * 0.998f) cur = t, best = c, changed = true;
                    }
                }
            }
            if (rc != DWT2_OK) return rc;
        }
    }
    *choice = best;
    return tune_apply(p, best);
}

int dwt2_inverse(dwt2_plan_t p, const void* coef, void* out, void* workspace, void* stream) {
    return run_inverse_like(p, coef, out, workspace, stream, false);
}

int dwt2_adjoint(dwt2_plan_t p, const void* coef_grad, void* in_grad, void* workspace, void* stream) {
    return run_inverse_like(p, coef_grad, in_grad, workspace, stream, true);
}

int dwt2_adjoint_l1(dwt2_plan_t p, const void* coef, void* in_grad, float scale, void* workspace, void* stream) {
    return run_inverse_like(p, coef, in_grad, workspace, stream, true, true, scale);
}

int dwt2_adjoint_l1_dev(dwt2_plan_t p, const void* coef, void* in_grad, const float* scale_dev, float scale,
                        void* workspace, void* stream) {
    if (!scale_dev) return DWT2_ERR_INVALID_ARG;
    return run_inverse_like(p, coef, in_grad, workspace, stream, true, true, scale, scale_dev);
}

}  // extern "C"

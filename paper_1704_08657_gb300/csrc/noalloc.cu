// noalloc.cu -- dwt2_forward_noalloc: the forward pyramid of one image with no
// device allocation at all, for callers that cannot allocate device memory
// when they transform: code that runs while a CUDA graph is being captured in
// a mode that forbids cudaMalloc, real-time pipelines that allow no
// allocation after start-up, and plug-ins whose host application owns all
// device memory and gives them no allocator.  A plan (dwt2_plan) allocates a
// status word and the multi-level forward needs a caller workspace; this entry
// point needs neither.
//
// The intermediate low-low bands of levels 1 .. L-1 live in one file-scope
// device array of NOALLOC_SCRATCH_BYTES (32 MiB).  Every GPU that loads the
// library holds that array until the process exits.  Every call shares it and
// it keeps the last call's contents; nothing in it has to start at zero
// (each call writes every element before reading it).  Calls whose work
// overlaps on the GPU (two streams, or two host threads on one stream
// without ordering) race on the array.  A second file-scope word is the
// status word of these calls: a bounded device wait that runs out sets it,
// and dwt2_noalloc_status reads and clears it (it starts at zero when the
// library is loaded).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/dwt2.h"
#include "internal.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;
constexpr int NOALLOC_MAX_DEVICES = 64;

// The scratch.  In host code this name is only a host-side stand-in for the
// device array; kernels get the device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
static __device__ unsigned g_noalloc_status;

struct NoallocDevice {
    bool ready;
    void* scratch;     // device address of g_noalloc_scratch on this device
    unsigned* status;  // device address of g_noalloc_status on this device
    uint64_t timeout_ns;
    int sm_count;
    int fwd_bps[4][3];  // resident forward blocks per SM by coefficient type and scheme
};

std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[NOALLOC_MAX_DEVICES];

// Set-up, once per device, with that device current: the device addresses
// of the scratch array and the status word, the SM count and the bounded-wait
// limit (DWT2_TIMEOUT_MS, as for plans; read once).
int noalloc_setup(int dev, NoallocDevice** out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return DWT2_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice& d = g_noalloc_dev[dev];
    if (!d.ready) {
        void* ptr = nullptr;
        void* sptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr ||
            cudaGetSymbolAddress(&sptr, g_noalloc_status) != cudaSuccess || sptr == nullptr) {
            cudaGetLastError();
            return DWT2_ERR_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return DWT2_ERR_CUDA;
        }
        d.scratch = ptr;
        d.status = static_cast<unsigned*>(sptr);
        const char* tm = getenv("DWT2_TIMEOUT_MS");
        const int ms = (tm && *tm) ? atoi(tm) : 2000;
        d.timeout_ns = uint64_t(ms > 0 ? ms : 2000) * 1000000ull;
        d.sm_count = sms;
        for (int dt = 0; dt < 4; ++dt)
            for (int sc = 0; sc < 3; ++sc)
                d.fwd_bps[dt][sc] = dwt2::forward_blocks_per_sm(dt == DWT2_I32 ? DWT2_CDF53_INT : DWT2_CDF97, sc, dt,
                                                               dwt2::FWD_CFGS[0]);
        d.ready = true;
    }
    *out = &d;
    return DWT2_OK;
}

typedef CUresult (*NoallocEncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                    CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                    CUtensorMapFloatOOBfill);

NoallocEncodeFn noalloc_encoder() {
    static NoallocEncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<NoallocEncodeFn>(p);
    });
    return fn;
}

int noalloc_map(CUtensorMap* m, const void* base, int w, int h, int64_t pitch, int box_w, int box_rows,
                bool is_int) {
    NoallocEncodeFn enc = noalloc_encoder();
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

int64_t noalloc_round4(int64_t v) { return (v + 3) / 4 * 4; }
size_t noalloc_align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

extern "C" int dwt2_forward_noalloc(int wavelet, int levels, int scheme, int coef_dtype, int h, int w,
                                    int64_t pitch_elems, const void* in, void* coef, void* stream) {
    using namespace dwt2;
    if (!in || !coef || levels < 1 || levels > 30 || h < 1 || w < 1 || pitch_elems < w)
        return DWT2_ERR_INVALID_ARG;
    if (wavelet != DWT2_CDF97 && wavelet != DWT2_CDF53_INT) return DWT2_ERR_INVALID_ARG;
    if (scheme < DWT2_NONSEP || scheme > DWT2_SEP_LIFTING) return DWT2_ERR_INVALID_ARG;
    if (coef_dtype < DWT2_F32 || coef_dtype > DWT2_I32) return DWT2_ERR_INVALID_ARG;
    if (wavelet == DWT2_CDF97 && coef_dtype == DWT2_I32) return DWT2_ERR_UNSUPPORTED;
    if (wavelet == DWT2_CDF53_INT && (coef_dtype != DWT2_I32 || scheme == DWT2_NONSEP_REDUCED))
        return DWT2_ERR_UNSUPPORTED;
    if (pitch_elems % 4 != 0 || reinterpret_cast<uintptr_t>(in) % 16 != 0) return DWT2_ERR_MISALIGNED;
    const size_t csz = (coef_dtype == DWT2_F16 || coef_dtype == DWT2_BF16) ? 2 : 4;
    if (reinterpret_cast<uintptr_t>(coef) % csz != 0) return DWT2_ERR_MISALIGNED;

    // level geometry and the scratch layout (two ping-pong low-low buffers)
    int lh[32], lw[32];
    {
        int hh = h, ww = w;
        for (int l = 0; l < levels; ++l) {
            if (hh < 2 || ww < 2) return DWT2_ERR_LEVELS_TOO_DEEP;
            lh[l] = hh;
            lw[l] = ww;
            hh = (hh + 1) / 2;
            ww = (ww + 1) / 2;
        }
    }
    size_t need[2] = {0, 0};
    for (int l = 0; l + 1 < levels; ++l) {
        const size_t b = size_t((lh[l] + 1) / 2) * size_t(noalloc_round4((lw[l] + 1) / 2)) * 4;
        need[l % 2] = std::max(need[l % 2], b);
    }
    const size_t off1 = noalloc_align256(need[0]);
    if (off1 + noalloc_align256(need[1]) > NOALLOC_SCRATCH_BYTES) return DWT2_ERR_TOO_LARGE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DWT2_ERR_CUDA;
    }
    NoallocDevice* st = nullptr;
    int rc = noalloc_setup(dev, &st);
    if (rc != DWT2_OK) return rc;
    char* scratch = static_cast<char*>(st->scratch);
    char* buf[2] = {scratch, scratch + off1};

    const bool is_int = wavelet == DWT2_CDF53_INT;
    const FwdCfg cfg = FWD_CFGS[0];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int l = 0; l < levels; ++l) {
        const int H = lh[l], W = lw[l];
        const void* src = (l == 0) ? in : static_cast<const void*>(buf[(l - 1) % 2]);
        const int64_t src_pitch = (l == 0) ? pitch_elems : noalloc_round4(W);  // = round4(wq of level l-1)
        CUtensorMap box, row;
        rc = noalloc_map(&box, src, W, H, src_pitch, fwd_strip_px(cfg), 2 * cfg.qr, is_int);
        if (rc == DWT2_OK) rc = noalloc_map(&row, src, W, H, src_pitch, fwd_strip_px(cfg), 1, is_int);
        if (rc != DWT2_OK) return rc;
        FwdParams fp{};  // no inter-level overlap: every level waits for the previous grid
        fp.h = H, fp.w = W, fp.hq = (H + 1) / 2, fp.wq = (W + 1) / 2, fp.hh = H / 2, fp.wh = W / 2;
        // segments of the height dwt2_forward chooses (rounds x (rows + 4) minimal)
        fp.n_strips = (fp.wq + fwd_out_quads(cfg, wavelet) - 1) / fwd_out_quads(cfg, wavelet);
        {
            const int64_t max_warps =
                int64_t(st->sm_count) * std::max(st->fwd_bps[coef_dtype][scheme], 1) * cfg.nw;
            int best = std::min(48, fp.hq);
            int64_t best_cost = INT64_MAX;
            for (int seg = std::min(8, fp.hq); seg <= std::min(48, fp.hq); ++seg) {
                const int64_t units = int64_t((fp.hq + seg - 1) / seg) * fp.n_strips;
                const int64_t cost = ((units + max_warps - 1) / max_warps) * (seg + 4);
                if (cost < best_cost) best_cost = cost, best = seg;
            }
            fp.seg_rows = best;
        }
        fp.n_segs = (fp.hq + fp.seg_rows - 1) / fp.seg_rows;
        fp.n_units = fp.n_segs * fp.n_strips;
        fp.balanced = 0;
        fp.pdl = 0;
        const int grid = (fp.n_units + cfg.nw - 1) / cfg.nw;
        fp.coef = coef;
        fp.coef_pitch = pitch_elems;
        const bool last = (l == levels - 1);
        if (last) {
            fp.ll = coef;
            fp.ll_pitch = pitch_elems;
            fp.ll_is_ct = 0;
        } else {
            fp.ll = buf[l % 2];
            fp.ll_pitch = noalloc_round4(fp.wq);
            fp.ll_is_ct = 1;
        }
        const bool coef_vec = (pitch_elems % 2 == 0) && (reinterpret_cast<uintptr_t>(coef) % (2 * csz) == 0);
        fp.vec_lo = coef_vec;
        fp.vec_hi = coef_vec && (fp.wq % 2 == 0);
        fp.vec_ll = last ? coef_vec : 1;
        fp.status = st->status;
        fp.timeout_ns = st->timeout_ns;
        int e;
        switch (coef_dtype) {
            case DWT2_F32: e = launch_forward_f32(wavelet, scheme, box, row, fp, grid, cfg, s); break;
            case DWT2_F16: e = launch_forward_f16(wavelet, scheme, box, row, fp, grid, cfg, s); break;
            case DWT2_BF16: e = launch_forward_bf16(wavelet, scheme, box, row, fp, grid, cfg, s); break;
            default: e = launch_forward_i32(wavelet, scheme, box, row, fp, grid, cfg, s); break;
        }
        if (e != cudaSuccess) return DWT2_ERR_CUDA;
    }
    return DWT2_OK;
}

// The status word of dwt2_forward_noalloc on the current device: wait for the
// stream, read the word and clear it.  Copies through no caller or library
// allocation (a four-byte read into a local variable, a four-byte clear).
extern "C" int dwt2_noalloc_status(void* stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DWT2_ERR_CUDA;
    }
    NoallocDevice* st = nullptr;
    const int rc = noalloc_setup(dev, &st);
    if (rc != DWT2_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned h = 0;
    if (cudaMemcpyAsync(&h, st->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaMemsetAsync(st->status, 0, sizeof(unsigned), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return DWT2_ERR_CUDA;
    }
    if (h & dwt2::DEV_TIMEOUT) return DWT2_ERR_TIMEOUT;
    if (h & dwt2::DEV_CHECK) return DWT2_ERR_DEVICE_CHECK;
    return DWT2_OK;
}

// kernels.cuh -- the transform kernels of one pyramid level.
//
// Work decomposition: the level is cut into vertical strips of 32*QL - 4
// output quads (a warp loads 64*QL pixels; 4 on each side are halo) and
// horizontal segments of seg_rows output quad rows.  One (strip, segment)
// pair is a unit of work for one warp.  A warp streams the quad rows of its
// unit top to bottom through the row pipeline of the scheme (schemes.cuh),
// starting two quad rows above the segment (warm-up) and running LAG rows
// past it, in groups of PHASES arrivals unrolled at compile time.
//
// Forward: each warp owns a ring of NST shared-memory stages of QR quad rows
// (2*QR pixel rows x 64*QL pixels) filled by 2-D TMA loads that complete on
// one mbarrier per stage; lane 0 refills a stage once the warp has read it.
// Rows outside the image are fetched from their whole-sample mirror rows (one
// single-row TMA box per pixel row); columns outside the image are mirrored in
// shared memory by the edge strips.  With the symmetric extension in place the
// lifting needs no boundary cases: every step preserves the symmetry, so the
// exact per-step mirrored result appears inside the image.
//
// Inverse and adjoint: the four bands are read with vector loads, two quad
// rows ahead of the pipeline.  The inverse reads mirrored band positions at the
// edges (the extension of the coefficients that the symmetric image extension
// produces); the adjoint reads zeros there and applies the transposed boundary
// weights of Adj97 instead.
#pragma once

#include <type_traits>
#include <utility>

#include "schemes.cuh"

namespace dwt2 {

// compile-time loop: f(std::integral_constant<int, 0>) ... f(<N-1>)
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <class CT>
__device__ __forceinline__ void ld4_smem(const CT* p, CT* v) {
    if constexpr (std::is_same<CT, float>::value) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    } else {
        const int4 t = *reinterpret_cast<const int4*>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    }
}

template <class CT>
__device__ __forceinline__ void st4(CT* p, CT a, CT b, CT c, CT d) {
    if constexpr (std::is_same<CT, float>::value)
        *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
    else
        *reinterpret_cast<int4*>(p) = make_int4(a, b, c, d);
}

// The pieces of work of one warp, as (strip, first quad row, end quad row):
// balanced mode gives each warp one contiguous range of the strip-major quad
// rows (split where it crosses a strip end); otherwise fixed units of
// seg_rows rows are dealt round-robin.
template <class P>
struct Pieces {
    int64_t rb, re;
    int unit, stride;
    __device__ __forceinline__ Pieces(const P& p, int wg, int nwarps) {
        const int64_t T = int64_t(p.n_strips) * p.hq;
        rb = T * wg / nwarps;
        re = T * (wg + 1) / nwarps;
        unit = wg;
        stride = nwarps;
    }
    __device__ __forceinline__ bool next(const P& p, int& s, int& R0, int& R1) {
        if (p.balanced) {
            if (rb >= re) return false;
            s = int(rb / p.hq);
            R0 = int(rb - int64_t(s) * p.hq);
            R1 = int(min(int64_t(p.hq), R0 + (re - rb)));
            rb += R1 - R0;
            return true;
        }
        if (unit >= p.n_units) return false;
        s = unit % p.n_strips;
        R0 = (unit / p.n_strips) * p.seg_rows;
        R1 = min(R0 + p.seg_rows, p.hq);
        unit += stride;
        return true;
    }
};

// shared-memory bytes of a forward launch
template <int QL, int QR, int NST, int NW>
constexpr size_t fwd_smem_bytes() {
    return size_t(NW) * NST * (2 * QR * 64 * QL * 4) + size_t(NW) * NST * 8;
}

// One quad row (two pixel rows) of the lane from a shared-memory stage; edge
// strips replace pixels outside [0, w) by their mirror images.
template <class CT, int QL>
__device__ __forceinline__ void load_quad_row(const CT* s0, Row<CT, QL>& r, int lane, bool edge, int x0, int w) {
    constexpr int SPX = 64 * QL;
    const CT* s1 = s0 + SPX;
    CT e[2 * QL], o[2 * QL];
#pragma unroll
    for (int k = 0; k < 2 * QL; k += 4) {
        ld4_smem<CT>(s0 + 2 * QL * lane + k, e + k);
        ld4_smem<CT>(s1 + 2 * QL * lane + k, o + k);
    }
    if (edge) {
#pragma unroll
        for (int k = 0; k < 2 * QL; ++k) {
            const int px = x0 + 2 * QL * lane + k;
            if (px < 0 || px >= w) {
                const int src = fold_ws(px, w) - x0;
                const bool in = (src >= 0) && (src < SPX);
                e[k] = in ? s0[src] : CT(0);
                o[k] = in ? s1[src] : CT(0);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        r.c1[q] = e[2 * q];
        r.c2[q] = e[2 * q + 1];
        r.c3[q] = o[2 * q];
        r.c4[q] = o[2 * q + 1];
    }
}

// Edge strips of the forward: once a stage has landed, every pixel of the
// lane outside [0, w) takes the value of its whole-sample mirror in place
// (zero where the mirror lies outside the strip, beyond the filter support of
// any stored output).  Sources are pixels inside the image, which no lane
// rewrites, so the lanes need no barrier between them; the proxy fence orders
// these generic writes before the next asynchronous fill of the stage.  Not
// inlined: the row loop of interior strips stays as small as it was.
template <class CT, int QL>
__device__ __noinline__ void fwd_fix_edges(CT* stage, int rows, int x0, int w, int lane) {
    constexpr int SPX = 64 * QL;
    for (int k = 0; k < 2 * QL; ++k) {
        const int px = x0 + 2 * QL * lane + k;
        if (px >= 0 && px < w) continue;
        const int src = fold_ws(px, w) - x0;
        const bool in = (src >= 0) && (src < SPX);
        for (int r = 0; r < rows; ++r) {
            CT* row = stage + r * SPX;
            row[2 * QL * lane + k] = in ? row[src] : CT(0);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------------------------------ loaders
// A loader fills one shared-memory stage (2*QR pixel rows of 64*QL pixels,
// starting at pixel column x0 and pixel row y0 of the level's input) and
// makes it complete on the stage's mbarrier.  Rows outside [0, h) are taken
// from their whole-sample mirror rows; columns outside [0, w) are left as
// zeros (load_quad_row mirrors them).

// 2-D TMA (cp.async.bulk.tensor) issued by lane 0; one box when every row is
// inside the image, else one single-row box per pixel row.
struct TmaLoader {
    static constexpr unsigned ARRIVALS = 1;
    const CUtensorMap* box;
    const CUtensorMap* row;
    template <class CT, int QL, int QR>
    __device__ __forceinline__ void issue(CT* dst, uint64_t* bar, int x0, int y0, int h, int /*w*/,
                                          int lane) const {
        constexpr int SPX = 64 * QL, ROWS = 2 * QR;
        if (lane != 0) return;
        mbar_expect_tx(bar, unsigned(ROWS * SPX * 4));
        if (y0 >= 0 && y0 + ROWS <= h) {
            tma_load_2d(dst, box, x0, y0, bar);
        } else {
#pragma unroll 1
            for (int r = 0; r < ROWS; ++r) tma_load_2d(dst + r * SPX, row, x0, fold_ws(y0 + r, h), bar);
        }
    }
};

// 16-byte cp.async by every lane (one 4-pixel chunk per lane per row and QL/2
// chunks per lane), zero-filling the part of a chunk past the right edge; each
// lane's copies arrive on the mbarrier when they land.  Needs a 16-byte
// aligned source row (pitch a multiple of 4 elements).
template <class CT>
struct CpAsyncLoader {
    static constexpr unsigned ARRIVALS = 32;
    const CT* src;
    int64_t pitch;
    template <class CT_, int QL, int QR>
    __device__ __forceinline__ void issue(CT_* dst, uint64_t* bar, int x0, int y0, int h, int w, int lane) const {
        constexpr int SPX = 64 * QL, ROWS = 2 * QR;
        const bool inside = (y0 >= 0) && (y0 + ROWS <= h);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const int y = inside ? y0 + r : fold_ws(y0 + r, h);
            const CT* srow = src + int64_t(y) * pitch;
#pragma unroll
            for (int k = 0; k < QL / 2; ++k) {
                const int c = lane + 32 * k;  // chunk index in the strip
                const int px = x0 + 4 * c;
                const int n = (px >= 0) ? max(0, min(4, w - px)) : 0;
                const CT* g = srow + (n > 0 ? px : 0);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst + r * SPX + 4 * c)),
                             "l"(g), "r"(4 * n)
                             : "memory");
            }
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
    }
};

// ------------------------------------------------------------------ forward
// One unit of work: quad rows [R0, R1) of strip s of one level.  P provides
// the level's geometry and outputs (fields of FwdParams); bufs / bars are the
// warp's stage ring, gstage the warp's running stage count (slot and mbarrier
// phase).  Returns false when a stage wait timed out.
//
// MODE 0 handles every strip.  MODE 1 and 2 are compiled for strips whose
// band rows all take paired stores (fwd_pairs_ok), with the low-low band in
// the compute type (1) or the coefficient type (2): their row loop has no
// store-alignment branches, which keeps the hot loop small in the instruction
// cache.  Edge strips run the same row loop as interior ones: their mirrored
// columns are filled in the stage (fwd_fix_edges) and per-lane masks drop the
// quads outside the bands.
template <class P>
__device__ __forceinline__ bool fwd_pairs_ok(const P& p, int x0, int QL, int halo) {
    // every pair starts at an even quad: with both band widths even no pair
    // straddles a band's last column; otherwise the strip must end inside both
    return p.vec_lo && p.vec_hi && (p.ll_is_ct || p.vec_ll) &&
           ((p.wq % 2 == 0 && p.wh % 2 == 0) || (x0 / 2 + 32 * QL - halo <= p.wh));
}

template <class Pipe, class OutT, int QL, int QR, int NST, int MODE = 0, class P, class Loader>
__device__ __forceinline__ bool fwd_unit(const P& p, const Loader& ld, int s, int R0, int R1,
                                         typename Pipe::CT* bufs, uint64_t* bars, uint32_t& gstage, int lane) {
    using CT = typename Pipe::CT;
    using R = Row<CT, QL>;
    constexpr int SPX = 64 * QL;
    constexpr int HQ = PipeGeom<Pipe>::HALO, WARM = PipeGeom<Pipe>::WARM;
    constexpr int OUTQ = 32 * QL - 2 * HQ;
    constexpr int ROWS = 2 * QR;
    constexpr int STAGE_ELEMS = ROWS * SPX;
    static_assert(PHASES % QR == 0, "a group of arrivals must cover whole stages");
    static_assert(QL % 2 == 0, "band stores go in pairs");

    const int A0 = R0 - WARM;                         // first quad row streamed
    const int n_arr = (R1 - R0) + WARM + Pipe::LAG;   // quad rows streamed
    const int n_grp = (n_arr + PHASES - 1) / PHASES;  // groups of arrivals (the last may stop early)
    const int NT = (n_arr + QR - 1) / QR;             // stages
    const int x0 = s * (2 * OUTQ) - 2 * HQ;           // first pixel (multiple of 4)
    const int jb = x0 / 2 + QL * lane;                // first quad column of the lane
    constexpr bool SPEC = MODE != 0;
    const bool edge = (x0 < 0) || (x0 + SPX > p.w);
    const bool llct = MODE == 1 ? true : (MODE == 2 ? false : bool(p.ll_is_ct));

    // which of the lane's quads this strip outputs, per band parity
    bool ev[QL], dv[QL], mp[QL];
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const int lq = QL * lane + q;
        mp[q] = (lq >= HQ) && (lq < 32 * QL - HQ);
        ev[q] = mp[q] && (jb + q < p.wq);
        dv[q] = mp[q] && (jb + q < p.wh);
    }
    // paired stores: both quads of the pair output by this strip and inside
    // the even-column (LL, LH) or odd-column (HL, HH) bands
    bool pe[QL / 2], po[QL / 2];
#pragma unroll
    for (int q = 0; q < QL; q += 2) {
        pe[q / 2] = mp[q] && mp[q + 1] && (jb + q + 1 < p.wq);
        po[q / 2] = mp[q] && mp[q + 1] && (jb + q + 1 < p.wh);
    }
    // warp-uniform: every band row takes paired stores
    const bool fast = SPEC ? true : fwd_pairs_ok(p, x0, QL, HQ);
    // band pointers at output row R0, advanced one pitch per stored row
    OutT* hl = reinterpret_cast<OutT*>(p.coef) + int64_t(R0) * p.coef_pitch + p.wq + jb;
    OutT* lh = reinterpret_cast<OutT*>(p.coef) + int64_t(p.hq + R0) * p.coef_pitch + jb;
    OutT* hh = lh + p.wq;
    CT* llc = reinterpret_cast<CT*>(p.ll) + int64_t(R0) * p.ll_pitch + jb;
    OutT* llo = reinterpret_cast<OutT*>(p.ll) + int64_t(R0) * p.ll_pitch + jb;

    for (int t = 0; t < NST && t < NT; ++t) {
        const uint32_t gs = gstage + t;
        ld.template issue<CT, QL, QR>(bufs + (gs % NST) * STAGE_ELEMS, &bars[gs % NST], x0, 2 * (A0 + t * QR), p.h,
                                      p.w, lane);
    }

    Pipe pipe;
    pipe.init();
    bool ok = true;
    int t = 0, slot = 0;
    const CT* stage = bufs;
    for (int gi = 0; gi < n_grp && ok; ++gi) {
        static_for<PHASES>([&](auto ph) {
            constexpr int PH = decltype(ph)::value;
            constexpr int QI = PH % QR;
            if (gi * PHASES + PH >= QR * NT) return;  // past the unit's last stage
            if constexpr (QI == 0) {
                if (!ok) return;
                const uint32_t gs = gstage + t;
                slot = gs % NST;
                if (!mbar_wait_bounded(&bars[slot], (gs / NST) & 1u, p.status, p.timeout_ns)) {
                    // give the copies still in flight a bounded time to land
                    for (int u = t + 1; u < NT && u < t + NST; ++u) {
                        const uint32_t gu = gstage + u;
                        mbar_wait_bounded(&bars[gu % NST], (gu / NST) & 1u, nullptr, p.timeout_ns);
                    }
                    ok = false;
                    return;
                }
                stage = bufs + slot * STAGE_ELEMS;
                if (edge) fwd_fix_edges<CT, QL>(const_cast<CT*>(stage), ROWS, x0, p.w, lane);
            }
            const int vi = A0 + gi * PHASES + PH;  // quad row streamed now
            load_quad_row<CT, QL>(stage + (2 * QI) * SPX, pipe.template slot<PH>(), lane, false, x0, p.w);
            const R& out = pipe.template step<PH>(vi);
            const int oi = vi - Pipe::LAG;
            const bool row_on = (oi >= R0) & (oi < R1);
            const bool orow = row_on & (oi < p.hh);
            if (fast) {
#pragma unroll
                for (int q = 0; q < QL; q += 2) {
                    const bool on_e = row_on & pe[q / 2], on_o = row_on & po[q / 2];
                    const bool oo_e = orow & pe[q / 2], oo_o = orow & po[q / 2];
                    if (llct) {
                        if (on_e) st_pair<CT>(llc + q, out.c1[q], out.c1[q + 1]);
                    } else {
                        if (on_e) st_pair<OutT>(llo + q, Cvt<OutT>::to(out.c1[q]), Cvt<OutT>::to(out.c1[q + 1]));
                    }
                    if (on_o) st_pair<OutT>(hl + q, Cvt<OutT>::to(out.c2[q]), Cvt<OutT>::to(out.c2[q + 1]));
                    if (oo_e) st_pair<OutT>(lh + q, Cvt<OutT>::to(out.c3[q]), Cvt<OutT>::to(out.c3[q + 1]));
                    if (oo_o) st_pair<OutT>(hh + q, Cvt<OutT>::to(out.c4[q]), Cvt<OutT>::to(out.c4[q + 1]));
                }
            } else if (row_on) {
#pragma unroll
                for (int q = 0; q < QL; q += 2) {
                    if (llct)
                        store_pair<CT, CT>(llc, q, out.c1[q], out.c1[q + 1], ev[q], ev[q + 1], true);
                    else
                        store_pair<OutT, CT>(llo, q, out.c1[q], out.c1[q + 1], ev[q], ev[q + 1], p.vec_ll);
                    store_pair<OutT, CT>(hl, q, out.c2[q], out.c2[q + 1], dv[q], dv[q + 1], p.vec_hi);
                    if (orow) {
                        store_pair<OutT, CT>(lh, q, out.c3[q], out.c3[q + 1], ev[q], ev[q + 1], p.vec_lo);
                        store_pair<OutT, CT>(hh, q, out.c4[q], out.c4[q + 1], dv[q], dv[q + 1], p.vec_hi);
                    }
                }
            }
            const int64_t cstep = row_on ? p.coef_pitch : 0;
            const int64_t lstep = row_on ? p.ll_pitch : 0;
            hl += cstep;
            lh += cstep;
            hh += cstep;
            llc += lstep;
            llo += lstep;
            if constexpr (QI == QR - 1) {
                __syncwarp();
                if (ok && t + NST < NT)
                    ld.template issue<CT, QL, QR>(bufs + slot * STAGE_ELEMS, &bars[slot], x0,
                                                  2 * (A0 + (t + NST) * QR), p.h, p.w, lane);
                ++t;
            }
        });
    }
    if (ok) gstage += NT;
    return ok;
}

template <class CT, int QL, int QR, int NST, int NW>
__device__ __forceinline__ void stage_ring(unsigned char* smem, int warp, CT*& bufs, uint64_t*& bars) {
    constexpr int STAGE_ELEMS = 2 * QR * 64 * QL;
    bufs = reinterpret_cast<CT*>(smem) + warp * NST * STAGE_ELEMS;
    bars = reinterpret_cast<uint64_t*>(smem + size_t(NW) * NST * STAGE_ELEMS * 4) + warp * NST;
}

// Inter-level overlap.  A unit of quad rows [R0, R1) streams input rows
// 2*R0-4 .. 2*(R1+LAG+QR-2)+1 (warm-up, pipeline lag, stage rounding), folded
// into [0, h) by the symmetric extension; lane 0 waits (bounded) until every
// previous-level segment holding such a row has all its strips complete, then
// orders its later TMA reads after what it observed.
template <int LAG, int QR, int WARM>
__device__ __forceinline__ bool fwd_wait_inputs(const FwdParams& p, int R0, int R1, int lane) {
    bool ok = true;
    if (lane == 0) {
        int lo = max(0, 2 * (R0 - WARM));
        const int end = 2 * (R1 + LAG + QR - 2) + 2;  // one past the last streamed row
        const int hi = min(p.h, end);
        if (end > p.h) lo = max(0, min(lo, 2 * p.h - 1 - end));  // mirrored rows past the bottom
        for (int g = lo / p.dep_seg; g <= (hi - 1) / p.dep_seg && ok; ++g) {
            const unsigned* c = p.dep_ctr + g;
            if (ld_acquire(c) >= unsigned(p.dep_need)) continue;
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire(c) < unsigned(p.dep_need)) {
                if (globaltimer_ns() - t0 > p.timeout_ns) {
                    ok = false;
                    break;
                }
                __nanosleep(128);
            }
        }
        if (!ok && p.status) atomicOr(p.status, DEV_TIMEOUT);
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    return __shfl_sync(FULL, ok ? 1 : 0, 0) != 0;
}

// after a unit's stores: count the unit in its segment with a release
// reduction (the warp barrier orders every lane's stores before lane 0's
// release); the consumer acquires the count and fences its async proxy
__device__ __forceinline__ void fwd_signal(unsigned* ctr, int lane) {
    __syncwarp();
    if (lane == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
}

// One pyramid level, TMA-fed: the warps take their units from Pieces.  SPEC
// compiles the specialised row loops for interior strips as well.
// Register budget of the forward kernels: the lifting pipelines in 4-warp
// blocks are held to five resident blocks per SM (at most 102 registers; the
// 5-level 16384^2 pyramid measured ~1 % faster than with four), the other
// pipelines and block sizes are left to the compiler.
template <class Pipe, int NW>
struct FwdMinBlocks {
    static constexpr int value = 1;
};
template <int S, int QL>
struct FwdMinBlocks<Fwd97<S, QL>, 4> {
    static constexpr int value = 5;
};
template <int S, int QL>
struct FwdMinBlocks<Fwd53<S, QL>, 4> {
    static constexpr int value = 5;
};

template <class Pipe, class OutT, int QL, int QR, int NST, int NW, bool SPEC>
__global__ void __launch_bounds__(NW * 32, FwdMinBlocks<Pipe, NW>::value)
    fwd_tma_kernel(const __grid_constant__ CUtensorMap tm_box, const __grid_constant__ CUtensorMap tm_row,
                   const FwdParams p) {
    using CT = typename Pipe::CT;
    constexpr int HQ = PipeGeom<Pipe>::HALO;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CT* bufs;
    uint64_t* bars;
    stage_ring<CT, QL, QR, NST, NW>(smem, warp, bufs, bars);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NST; ++i) mbar_init(&bars[i], TmaLoader::ARRIVALS);
        fence_mbar_init();
        tma_prefetch_desc(&tm_box);
        tma_prefetch_desc(&tm_row);
    }
    __syncwarp();
    // the input (the previous level's low-low band) and the outputs are only
    // touched after the previous grid in the stream has completed, or, with
    // inter-level overlap, after the segments a unit reads are complete
    if (p.dep_ctr == nullptr) griddep_wait();
    griddep_launch_dependents();
    const TmaLoader ld{&tm_box, &tm_row};
    uint32_t gstage = 0;
    Pieces<FwdParams> pieces(p, blockIdx.x * NW + warp, gridDim.x * NW);
    int s, R0, R1;
    while (pieces.next(p, s, R0, R1)) {
        if (p.dep_ctr != nullptr && !fwd_wait_inputs<Pipe::LAG, QR, PipeGeom<Pipe>::WARM>(p, R0, R1, lane)) return;
        bool ok;
        if constexpr (SPEC) {
            if (fwd_pairs_ok(p, s * (2 * (32 * QL - 2 * HQ)) - 2 * HQ, QL, HQ))
                ok = p.ll_is_ct ? fwd_unit<Pipe, OutT, QL, QR, NST, 1>(p, ld, s, R0, R1, bufs, bars, gstage, lane)
                                : fwd_unit<Pipe, OutT, QL, QR, NST, 2>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
            else
                ok = fwd_unit<Pipe, OutT, QL, QR, NST, 0>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
        } else {
            ok = fwd_unit<Pipe, OutT, QL, QR, NST, 0>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
        }
        if (!ok) return;
        if (p.out_ctr != nullptr && !(p.test_drop && s == 0 && R0 == 0)) fwd_signal(p.out_ctr + R0 / p.seg_rows, lane);
    }
}

// One level of a group of images (GroupLaunch): the warps take units in order,
// find their image by a binary search over the group's unit ranges, and run
// the single-image row loop with that image's parameters and tensor maps.
// Launches of one level touch disjoint images, so only the first launch of a
// level waits for what came before it; the others start as soon as the
// previous launch has placed all its blocks.
template <class Pipe, class OutT, int QL, int QR, int NST, int NW, bool SPEC>
__global__ void __launch_bounds__(NW * 32, FwdMinBlocks<Pipe, NW>::value)
    fwd_group_kernel(const __grid_constant__ GroupLaunch L) {
    using CT = typename Pipe::CT;
    constexpr int HQ = PipeGeom<Pipe>::HALO;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CT* bufs;
    uint64_t* bars;
    stage_ring<CT, QL, QR, NST, NW>(smem, warp, bufs, bars);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NST; ++i) mbar_init(&bars[i], TmaLoader::ARRIVALS);
        fence_mbar_init();
    }
    __syncwarp();
    if (L.wait_prev) griddep_wait();
    griddep_launch_dependents();
    uint32_t gstage = 0;
    const int stride = gridDim.x * NW;
    for (int u = blockIdx.x * NW + warp; u < L.n_units; u += stride) {
        int lo = 0, hi = L.n_img - 1;  // the last image whose u_begin <= u
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.img[mid].u_begin <= u) lo = mid;
            else hi = mid - 1;
        }
        const FwdParams& p = L.img[lo].p;
        const int lu = u - L.img[lo].u_begin;
        const int s = lu % p.n_strips;
        const int R0 = (lu / p.n_strips) * p.seg_rows;
        const int R1 = min(R0 + p.seg_rows, p.hq);
        const TmaLoader ld{&L.maps[2 * lo], &L.maps[2 * lo + 1]};
        if (lane == 0) {
            tma_prefetch_desc(ld.box);
            tma_prefetch_desc(ld.row);
        }
        bool ok;
        if constexpr (SPEC) {
            if (fwd_pairs_ok(p, s * (2 * (32 * QL - 2 * HQ)) - 2 * HQ, QL, HQ))
                ok = p.ll_is_ct ? fwd_unit<Pipe, OutT, QL, QR, NST, 1>(p, ld, s, R0, R1, bufs, bars, gstage, lane)
                                : fwd_unit<Pipe, OutT, QL, QR, NST, 2>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
            else
                ok = fwd_unit<Pipe, OutT, QL, QR, NST, 0>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
        } else {
            ok = fwd_unit<Pipe, OutT, QL, QR, NST, 0>(p, ld, s, R0, R1, bufs, bars, gstage, lane);
        }
        if (!ok) return;
    }
}

// ------------------------------------------------- persistent (batched) forward
// All units of all images and levels of a plan in one launch.  Units are taken
// from a device queue in the plan's order; a unit of level l first waits
// (bounded) until the level l-1 segments it reads are complete, i.e. their
// counters reached the strip count; after its stores it bumps the counter of
// its own segment.  The queue order puts every unit about one GPU round behind
// the segments it depends on, so waits are rare and the low-low band it reads
// was written moments before (usually still in L2).

// the geometry and outputs of one unit's level, with the field names fwd_unit uses
struct PmlView {
    int h, w, hq, wq, hh, wh;
    void* coef;
    int64_t coef_pitch;
    void* ll;
    int64_t ll_pitch;
    int ll_is_ct;
    int vec_lo, vec_hi, vec_ll;
    unsigned* status;
    uint64_t timeout_ns;
};

template <class Pipe, class OutT, int QL, int QR, int NST, int NW, bool TMA>
__global__ void __launch_bounds__(NW * 32, FwdMinBlocks<Pipe, NW>::value) pml_kernel(const __grid_constant__ PmlLaunch L) {
    using CT = typename Pipe::CT;
    const PmlParams& P = L.base;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    CT* bufs;
    uint64_t* bars;
    stage_ring<CT, QL, QR, NST, NW>(smem, warp, bufs, bars);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NST; ++i) mbar_init(&bars[i], TMA ? TmaLoader::ARRIVALS : CpAsyncLoader<CT>::ARRIVALS);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t gstage = 0;
    for (;;) {
        int u = 0;
        if (lane == 0) u = int(atomicAdd(P.queue, 1u));
        u = __shfl_sync(FULL, u, 0);
        if (u >= P.n_units) break;
        const PmlUnit un = P.units[u];
        const PmlDesc& d = P.descs[un.desc];
        if (d.dep_base >= 0) {
            bool waited_ok = true;
            if (lane == 0) {
                for (int g = un.dep_lo; g <= un.dep_hi; ++g) {
                    const unsigned* c = P.counters + d.dep_base + g;
                    if (ld_acquire(c) >= unsigned(d.dep_need)) continue;
                    const uint64_t t0 = globaltimer_ns();
                    while (ld_acquire(c) < unsigned(d.dep_need)) {
                        if (globaltimer_ns() - t0 > P.timeout_ns) {
                            waited_ok = false;
                            break;
                        }
                        __nanosleep(256);
                    }
                }
                if (!waited_ok && P.status) atomicOr(P.status, DEV_TIMEOUT);
                // the level's input was written through the generic proxy by other
                // warps; TMA reads through the async proxy
                if (TMA) asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            __syncwarp();
        }
        PmlView v;
        v.h = d.h, v.w = d.w, v.hq = d.hq, v.wq = d.wq, v.hh = d.hh, v.wh = d.wh;
        v.coef = static_cast<OutT*>(P.coef) + d.coef_off;
        v.coef_pitch = d.coef_pitch;
        v.ll = d.ll_is_ct ? static_cast<void*>(static_cast<CT*>(P.ws) + d.ll_off)
                          : static_cast<void*>(static_cast<OutT*>(P.coef) + d.ll_off);
        v.ll_pitch = d.ll_pitch;
        v.ll_is_ct = d.ll_is_ct;
        v.vec_lo = d.vec_lo && P.coef_vec, v.vec_hi = d.vec_hi && P.coef_vec;
        v.vec_ll = d.ll_is_ct ? 1 : (d.vec_ll && P.coef_vec);
        v.status = P.status;
        v.timeout_ns = P.timeout_ns;
        const int R0 = un.g * d.seg_rows;
        const int R1 = min(R0 + d.seg_rows, d.hq);
        bool ok;
        if constexpr (TMA) {
            const TmaLoader ld{L.maps + 2 * un.desc, L.maps + 2 * un.desc + 1};
            if (lane == 0) {
                tma_prefetch_desc(ld.box);
                tma_prefetch_desc(ld.row);
            }
            ok = fwd_unit<Pipe, OutT, QL, QR, NST>(v, ld, un.s, R0, R1, bufs, bars, gstage, lane);
        } else {
            const CT* src = d.src_is_ws ? static_cast<const CT*>(P.ws) + d.src_off
                                        : static_cast<const CT*>(P.in) + d.src_off;
            const CpAsyncLoader<CT> ld{src, d.src_pitch};
            ok = fwd_unit<Pipe, OutT, QL, QR, NST>(v, ld, un.s, R0, R1, bufs, bars, gstage, lane);
        }
        if (!ok) return;
        // this unit's stores must be visible to the TMA reads of later units
        if (TMA) asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncwarp();
        if (lane == 0 && !(P.test_drop_signal && u == 0)) {
            __threadfence();
            atomicAdd(P.counters + d.ctr_base + un.g, 1u);
        }
    }
}

// ------------------------------------------------- band loads (inverse, adjoint)
template <class T>
__device__ __forceinline__ void ld_pair(const T* p, float& a, float& b, bool vec) {
    if (vec) {
        if constexpr (sizeof(T) == 4) {
            const float2 t = *reinterpret_cast<const float2*>(p);
            a = t.x, b = t.y;
        } else if constexpr (std::is_same<T, __half>::value) {
            const __half2 t = *reinterpret_cast<const __half2*>(p);
            a = __low2float(t), b = __high2float(t);
        } else {
            const __nv_bfloat162 t = *reinterpret_cast<const __nv_bfloat162*>(p);
            a = __low2float(t), b = __high2float(t);
        }
    } else {
        a = Cvt<T>::from(p[0]);
        b = Cvt<T>::from(p[1]);
    }
}
__device__ __forceinline__ void ld_pair(const int* p, int& a, int& b, bool vec) {
    if (vec) {
        const int2 t = *reinterpret_cast<const int2*>(p);
        a = t.x, b = t.y;
    } else {
        a = p[0];
        b = p[1];
    }
}

template <class T, class CT>
__device__ __forceinline__ CT ld_one(const T* p) {
    return CT(Cvt<T>::from(*p));
}

// One quad row of the lane's quads from the four bands.  MIRROR: positions
// outside the image read their mirror images; otherwise they read zero.
template <class CT, class BT, bool MIRROR, int QL>
__device__ __forceinline__ void load_bands(const InvParams& p, int vi, int jb, bool fast, Row<CT, QL>& r) {
    const BT* coef = reinterpret_cast<const BT*>(p.coef);
    if (fast) {  // whole strip and row inside the bands: direct pair loads
        const int64_t re = vi, ro = vi;
        const BT* hl = coef + re * p.coef_pitch + p.wq + jb;
        const BT* lh = coef + (p.hq + ro) * p.coef_pitch + jb;
        const BT* hh = lh + p.wq;
#pragma unroll
        for (int q = 0; q < QL; q += 2) {
            if (p.ll_is_ct) {
                const CT* ll = reinterpret_cast<const CT*>(p.ll) + re * p.ll_pitch + jb;
                ld_pair(ll + q, r.c1[q], r.c1[q + 1], p.vec_ll);
            } else {
                const BT* ll = reinterpret_cast<const BT*>(p.ll) + re * p.ll_pitch + jb;
                ld_pair(ll + q, r.c1[q], r.c1[q + 1], p.vec_ll);
            }
            ld_pair(hl + q, r.c2[q], r.c2[q + 1], p.vec_in_hi);
            ld_pair(lh + q, r.c3[q], r.c3[q + 1], p.vec_in_lo);
            ld_pair(hh + q, r.c4[q], r.c4[q + 1], p.vec_in_hi);
        }
        return;
    }
    int re, ro;
    bool rev, rov;
    if (MIRROR) {
        re = fold_ws(2 * vi, p.h) >> 1;
        ro = fold_ws(2 * vi + 1, p.h) >> 1;
        rev = rov = true;
    } else {
        rev = (vi >= 0) && (vi < p.hq);
        rov = (vi >= 0) && (vi < p.hh);
        re = rev ? vi : 0;
        ro = rov ? vi : 0;
    }
    // defensive clamps keep every address inside the bands
    re = min(max(re, 0), p.hq - 1);
    ro = min(max(ro, 0), max(p.hh - 1, 0));
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const int j = jb + q;
        int ce, co;
        bool cev, cov;
        if (MIRROR) {
            ce = fold_ws(2 * j, p.w) >> 1;
            co = fold_ws(2 * j + 1, p.w) >> 1;
            cev = cov = true;
        } else {
            cev = (j >= 0) && (j < p.wq);
            cov = (j >= 0) && (j < p.wh);
            ce = cev ? j : 0;
            co = cov ? j : 0;
        }
        ce = min(max(ce, 0), p.wq - 1);
        co = min(max(co, 0), max(p.wh - 1, 0));
        CT v1, v2, v3, v4;
        if (p.ll_is_ct)
            v1 = reinterpret_cast<const CT*>(p.ll)[int64_t(re) * p.ll_pitch + ce];
        else
            v1 = ld_one<BT, CT>(reinterpret_cast<const BT*>(p.ll) + int64_t(re) * p.ll_pitch + ce);
        v2 = ld_one<BT, CT>(coef + int64_t(re) * p.coef_pitch + p.wq + co);
        v3 = ld_one<BT, CT>(coef + int64_t(p.hq + ro) * p.coef_pitch + ce);
        v4 = ld_one<BT, CT>(coef + int64_t(p.hq + ro) * p.coef_pitch + p.wq + co);
        r.c1[q] = (rev && cev) ? v1 : CT(0);
        r.c2[q] = (rev && cov) ? v2 : CT(0);
        r.c3[q] = (rov && cev) ? v3 : CT(0);
        r.c4[q] = (rov && cov) ? v4 : CT(0);
    }
}

// L1 adjoint: the gradient of l1_scale * sum |detail| w.r.t. the coefficients
template <class CT, int QL>
__device__ __forceinline__ void l1_transform(const InvParams& p, Row<CT, QL>& r) {
    const float s = p.l1_scale_dev ? p.l1_scale * *p.l1_scale_dev : p.l1_scale;
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        if (!p.ll_is_ct) r.c1[q] = CT(0);  // the coarsest LL is not in the loss
        r.c2[q] = CT(r.c2[q] > 0 ? s : (r.c2[q] < 0 ? -s : 0.f));
        r.c3[q] = CT(r.c3[q] > 0 ? s : (r.c3[q] < 0 ? -s : 0.f));
        r.c4[q] = CT(r.c4[q] > 0 ? s : (r.c4[q] < 0 ? -s : 0.f));
    }
}

// --------------------------------------------------------- inverse / adjoint
// One unit (strip s, quad rows [R0, R1)) of one inverse or adjoint level.
// Pipe: Inv97<S, QL>, Inv53<S, QL> or Adj97<QL>.  BT: coefficient element type.
template <class Pipe, class BT, bool ADJ, int QL>
__device__ __forceinline__ void inv_unit(const InvParams& p, int s, int R0, int R1, int lane) {
    using CT = typename Pipe::CT;
    using R = Row<CT, QL>;
    constexpr bool MIRROR = !ADJ;
    constexpr int HQ = PipeGeom<Pipe>::HALO, WARM = PipeGeom<Pipe>::WARM;
    constexpr int OUTQ = 32 * QL - 2 * HQ;
    const int A0 = R0 - WARM;
    const int n_arr = (R1 - R0) + WARM + Pipe::LAG;
    const int n_grp = (n_arr + PHASES - 1) / PHASES;
    const int x0 = s * (2 * OUTQ) - 2 * HQ;
    const int jb = x0 / 2 + QL * lane;
    // the whole strip reads only existing band columns
    const bool fast_cols = (x0 >= 0) && (x0 / 2 + 32 * QL <= p.wh);
    bool mine[QL];
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const int lq = QL * lane + q;
        mine[q] = (lq >= HQ) && (lq < 32 * QL - HQ);
    }

    Pipe pipe;
    pipe.init();
    if constexpr (ADJ) {
#pragma unroll
        for (int q = 0; q < QL; ++q) pipe.hw[q] = axis_weights(jb + q, p.w);
        pipe.h = p.h;
    }
    auto fast_row = [&](int vi) { return fast_cols && vi >= 0 && 2 * vi + 1 < p.h; };

    R pf[2];  // rows vi+1 and vi+2 in flight
    load_bands<CT, BT, MIRROR, QL>(p, A0, jb, fast_row(A0), pf[0]);
    load_bands<CT, BT, MIRROR, QL>(p, A0 + 1, jb, fast_row(A0 + 1), pf[1]);
    if constexpr (ADJ) {
        if (p.l1) {
            l1_transform(p, pf[0]);
            l1_transform(p, pf[1]);
        }
    }
    CT* row_e = reinterpret_cast<CT*>(p.out) + int64_t(2 * R0) * p.out_pitch;
    const int px = 2 * jb;  // first pixel column of the lane
    for (int gi = 0; gi < n_grp; ++gi) {
        static_for<PHASES>([&](auto ph) {
            constexpr int PH = decltype(ph)::value;
            if (gi * PHASES + PH >= n_arr) return;
            const int vi = A0 + gi * PHASES + PH;
            pipe.template slot<PH>() = pf[PH % 2];
            load_bands<CT, BT, MIRROR, QL>(p, vi + 2, jb, fast_row(vi + 2), pf[PH % 2]);
            if constexpr (ADJ) {
                if (p.l1) l1_transform(p, pf[PH % 2]);
            }
            const R& out = pipe.template step<PH>(vi);
            const int oi = vi - Pipe::LAG;
            if (oi < R0 || oi >= R1) return;
            CT* row_o = row_e + p.out_pitch;
            const bool has_o = 2 * oi + 1 < p.h;
#pragma unroll
            for (int q = 0; q < QL; q += 2) {
                const int c = px + 2 * q;
                if (mine[q] && mine[q + 1] && p.vec_out && c + 3 < p.w) {
                    st4<CT>(row_e + c, out.c1[q], out.c2[q], out.c1[q + 1], out.c2[q + 1]);
                    if (has_o) st4<CT>(row_o + c, out.c3[q], out.c4[q], out.c3[q + 1], out.c4[q + 1]);
                } else {
                    const CT ev[4] = {out.c1[q], out.c2[q], out.c1[q + 1], out.c2[q + 1]};
                    const CT od[4] = {out.c3[q], out.c4[q], out.c3[q + 1], out.c4[q + 1]};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (mine[q + (k >> 1)] && c + k < p.w) {
                            row_e[c + k] = ev[k];
                            if (has_o) row_o[c + k] = od[k];
                        }
                    }
                }
            }
            row_e += 2 * p.out_pitch;
        });
    }
}

// cp.async of `bytes` (4 or 8) from global to shared memory; src_bytes 0
// zero-fills the destination.
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* dst, const void* src, bool valid) {
    static_assert(BYTES == 4 || BYTES == 8, "cp.async.ca copies 4, 8 or 16 bytes");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES),
                 "r"(valid ? BYTES : 0)
                 : "memory");
}

template <class T, class CT>
__device__ __forceinline__ void ld_pair_smem(const unsigned char* p, CT& a, CT& b) {
    if constexpr (std::is_same<T, float>::value) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        a = v.x, b = v.y;
    } else if constexpr (std::is_same<T, int>::value) {
        const int2 v = *reinterpret_cast<const int2*>(p);
        a = v.x, b = v.y;
    } else if constexpr (std::is_same<T, __half>::value) {
        const __half2 v = *reinterpret_cast<const __half2*>(p);
        a = __low2float(v), b = __high2float(v);
    } else {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(p);
        a = __low2float(v), b = __high2float(v);
    }
}

// Shared-memory ring of the staged inverse / adjoint: per stage QR quad rows
// of the four bands, 256 bytes per band row (the lane's two quads as one pair).
template <int QR, int NST, int NW>
constexpr size_t inv_smem_bytes() {
    return size_t(NW) * NST * QR * 4 * 256 + size_t(NW) * NST * 8;
}

// One unit of a strip: the bands stream through a ring of NST stages of QR
// quad rows filled by cp.async (mirrored rows for the inverse, zero rows for
// the adjoint at the top and bottom).  Interior strips copy each lane's quad
// pair at once; EDGE strips (the first and last of a row, 4-byte types) copy
// element by element from the mirrored (inverse) or zero-filled (adjoint)
// columns.  Returns false when a stage wait timed out.
template <class Pipe, class BT, bool ADJ, int QR, int NST, bool EDGE>
__device__ __forceinline__ bool inv_unit_staged(const InvParams& p, int s, int R0, int R1, int lane,
                                                unsigned char* ring, uint64_t* bars, uint32_t& gstage) {
    using CT = typename Pipe::CT;
    using R = Row<CT, 2>;
    constexpr int HQ = PipeGeom<Pipe>::HALO, WARM = PipeGeom<Pipe>::WARM;
    constexpr int QL = 2, OUTQ = 32 * QL - 2 * HQ;
    constexpr int BAND = 256, ROWB = 4 * BAND, STAGEB = QR * ROWB;
    constexpr int PB = 2 * int(sizeof(BT));  // bytes of a coefficient pair
    static_assert(PHASES % QR == 0, "a group of arrivals must cover whole stages");
    static_assert(HQ % 2 == 0, "a lane's two quads are both output or both halo");
    const int A0 = R0 - WARM;
    const int n_arr = (R1 - R0) + WARM + Pipe::LAG;
    const int n_grp = (n_arr + PHASES - 1) / PHASES;
    const int NT = (n_arr + QR - 1) / QR;
    const int x0 = s * (2 * OUTQ) - 2 * HQ;
    const int jb = x0 / 2 + QL * lane;
    const bool mine = (lane >= HQ / 2) && (lane < 32 - HQ / 2);
    const BT* coef = reinterpret_cast<const BT*>(p.coef);

    // EDGE: every lane copies its band elements one by one (4-byte types), at
    // the mirrored (inverse) or zero-filled (adjoint) columns
    int ce[2], co[2];
    bool cev[2], cov[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = jb + q;
        if (ADJ) {
            cev[q] = (j >= 0) && (j < p.wq);
            cov[q] = (j >= 0) && (j < p.wh);
            ce[q] = cev[q] ? j : 0;
            co[q] = cov[q] ? j : 0;
        } else {
            ce[q] = fold_ws(2 * j, p.w) >> 1;
            co[q] = fold_ws(2 * j + 1, p.w) >> 1;
            cev[q] = cov[q] = true;
        }
        ce[q] = min(max(ce[q], 0), p.wq - 1);
        co[q] = min(max(co[q], 0), max(p.wh - 1, 0));
    }

    auto issue = [&](int t, int slot) {
        unsigned char* st = ring + slot * STAGEB;
#pragma unroll
        for (int r = 0; r < QR; ++r) {
            const int vi = A0 + t * QR + r;
            int re, ro;
            bool rev, rov;
            if (ADJ) {
                rev = (vi >= 0) && (vi < p.hq);
                rov = (vi >= 0) && (vi < p.hh);
                re = rev ? vi : 0;
                ro = rov ? vi : 0;
            } else {
                const bool in = (vi >= 0) && (2 * vi + 1 < p.h);
                re = in ? vi : (fold_ws(2 * vi, p.h) >> 1);
                ro = in ? vi : (fold_ws(2 * vi + 1, p.h) >> 1);
                rev = rov = true;
            }
            unsigned char* d = st + r * ROWB;
            if constexpr (EDGE) {
                static_assert(sizeof(BT) == 4 && sizeof(CT) == 4, "element copies of 4-byte types");
                const CT* llr = reinterpret_cast<const CT*>(p.ll) + int64_t(re) * p.ll_pitch;
                const BT* hlr = coef + int64_t(re) * p.coef_pitch + p.wq;
                const BT* lhr = coef + int64_t(p.hq + ro) * p.coef_pitch;
                const BT* hhr = lhr + p.wq;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    cp_async_small<4>(d + lane * 8 + q * 4, llr + ce[q], rev && cev[q]);
                    cp_async_small<4>(d + BAND + lane * 8 + q * 4, hlr + co[q], rev && cov[q]);
                    cp_async_small<4>(d + 2 * BAND + lane * 8 + q * 4, lhr + ce[q], rov && cev[q]);
                    cp_async_small<4>(d + 3 * BAND + lane * 8 + q * 4, hhr + co[q], rov && cov[q]);
                }
            } else {
                if (p.ll_is_ct)
                    cp_async_small<8>(d + lane * 8, reinterpret_cast<const CT*>(p.ll) + int64_t(re) * p.ll_pitch + jb,
                                      rev);
                else
                    cp_async_small<PB>(d + lane * PB,
                                       reinterpret_cast<const BT*>(p.ll) + int64_t(re) * p.ll_pitch + jb, rev);
                cp_async_small<PB>(d + BAND + lane * PB, coef + int64_t(re) * p.coef_pitch + p.wq + jb, rev);
                cp_async_small<PB>(d + 2 * BAND + lane * PB, coef + int64_t(p.hq + ro) * p.coef_pitch + jb, rov);
                cp_async_small<PB>(d + 3 * BAND + lane * PB, coef + int64_t(p.hq + ro) * p.coef_pitch + p.wq + jb,
                                   rov);
            }
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&bars[slot]))
                     : "memory");
    };
    for (int t = 0; t < NST && t < NT; ++t) issue(t, (gstage + t) % NST);

    Pipe pipe;
    pipe.init();
    if constexpr (ADJ && !std::is_same<Pipe, AdjInner97<2>>::value) {
#pragma unroll
        for (int q = 0; q < QL; ++q) pipe.hw[q] = axis_weights(jb + q, p.w);
        pipe.h = p.h;
    }
    bool ok = true;
    int t = 0, slot = 0;
    const unsigned char* stage = ring;
    CT* row_e = reinterpret_cast<CT*>(p.out) + int64_t(2 * R0) * p.out_pitch;
    const int px = 2 * jb;
    for (int gi = 0; gi < n_grp && ok; ++gi) {
        static_for<PHASES>([&](auto ph) {
            constexpr int PH = decltype(ph)::value;
            constexpr int QI = PH % QR;
            if (gi * PHASES + PH >= QR * NT) return;
            if constexpr (QI == 0) {
                if (!ok) return;
                const uint32_t gs = gstage + t;
                slot = gs % NST;
                if (!mbar_wait_bounded(&bars[slot], (gs / NST) & 1u, p.status, p.timeout_ns)) {
                    for (int u = t + 1; u < NT && u < t + NST; ++u) {
                        const uint32_t gu = gstage + u;
                        mbar_wait_bounded(&bars[gu % NST], (gu / NST) & 1u, nullptr, p.timeout_ns);
                    }
                    ok = false;
                    return;
                }
                stage = ring + slot * STAGEB;
            }
            const int vi = A0 + gi * PHASES + PH;
            R& in = pipe.template slot<PH>();
            const unsigned char* d = stage + QI * ROWB;
            if (p.ll_is_ct)
                ld_pair_smem<CT, CT>(d + lane * 8, in.c1[0], in.c1[1]);
            else
                ld_pair_smem<BT, CT>(d + lane * PB, in.c1[0], in.c1[1]);
            ld_pair_smem<BT, CT>(d + BAND + lane * PB, in.c2[0], in.c2[1]);
            ld_pair_smem<BT, CT>(d + 2 * BAND + lane * PB, in.c3[0], in.c3[1]);
            ld_pair_smem<BT, CT>(d + 3 * BAND + lane * PB, in.c4[0], in.c4[1]);
            if constexpr (ADJ) {
                if (p.l1) l1_transform(p, in);
            }
            const R& out = pipe.template step<PH>(vi);
            const int oi = vi - Pipe::LAG;
            if (oi >= R0 && oi < R1) {
                CT* row_o = row_e + p.out_pitch;
                const bool has_o = 2 * oi + 1 < p.h;
                if (mine && p.vec_out && px + 3 < p.w) {
                    st4<CT>(row_e + px, out.c1[0], out.c2[0], out.c1[1], out.c2[1]);
                    if (has_o) st4<CT>(row_o + px, out.c3[0], out.c4[0], out.c3[1], out.c4[1]);
                } else if (mine) {
                    const CT ev[4] = {out.c1[0], out.c2[0], out.c1[1], out.c2[1]};
                    const CT od[4] = {out.c3[0], out.c4[0], out.c3[1], out.c4[1]};
#pragma unroll
                    for (int k2 = 0; k2 < 4; ++k2) {
                        if (px + k2 < p.w) {
                            row_e[px + k2] = ev[k2];
                            if (has_o) row_o[px + k2] = od[k2];
                        }
                    }
                }
                row_e += 2 * p.out_pitch;
            }
            if constexpr (QI == QR - 1) {
                __syncwarp();
                if (ok && t + NST < NT) issue(t + NST, slot);
                ++t;
            }
        });
    }
    if (ok) gstage += NT;
    return ok;
}

// inverse / adjoint unit: staged when every band row takes paired copies,
// else direct loads.  Adjoint units away from the boundary (every quad of
// the strip and every row the steps weight in [1, half - 2]) run the
// unweighted pipeline.  CLS selects the code compiled in: UNITS_INNER only the
// staged row loop of the inner units (inv_inner_rect), UNITS_EDGE every other
// path, UNITS_ALL both.
template <class Pipe, class BT, bool ADJ, int QR, int NST, int CLS = UNITS_ALL>
__device__ __forceinline__ bool inv_unit_any(const InvParams& p, int s, int R0, int R1, int lane,
                                             unsigned char* ring, uint64_t* bars, uint32_t& gstage) {
    using Inner = typename std::conditional<ADJ, AdjInner97<2>, Pipe>::type;
    if constexpr (CLS == UNITS_INNER) {
        return inv_unit_staged<Inner, BT, ADJ, QR, NST, false>(p, s, R0, R1, lane, ring, bars, gstage);
    } else {
        constexpr int HQ = PipeGeom<Pipe>::HALO;
        constexpr int OUTQ = 32 * 2 - 2 * HQ;
        const int x0 = s * (2 * OUTQ) - 2 * HQ;
        const bool staged = p.vec_in_lo && p.vec_in_hi && p.vec_ll;
        const bool interior = (x0 >= 0) && (x0 / 2 + 64 <= p.wh);
        if constexpr (ADJ && CLS == UNITS_ALL) {
            // the steps weight rows R0-4 .. R1+1 (see Adj97::step) and quads x0/2 .. x0/2+63
            const bool inner = staged && interior && (x0 / 2 >= 1) && (x0 / 2 + 63 <= p.wh - 2) && (R0 - 4 >= 1) &&
                               (R1 + 1 <= p.hh - 2);
            if (inner) return inv_unit_staged<Inner, BT, true, QR, NST, false>(p, s, R0, R1, lane, ring, bars, gstage);
        }
        if (staged && interior)
            return inv_unit_staged<Pipe, BT, ADJ, QR, NST, false>(p, s, R0, R1, lane, ring, bars, gstage);
        if constexpr (sizeof(BT) == 4) {
            if (staged) return inv_unit_staged<Pipe, BT, ADJ, QR, NST, true>(p, s, R0, R1, lane, ring, bars, gstage);
        }
        inv_unit<Pipe, BT, ADJ, 2>(p, s, R0, R1, lane);
        return true;
    }
}

template <int QR, int NST, int NW>
__device__ __forceinline__ void inv_ring(unsigned char* smem, int warp, int lane, unsigned char*& ring,
                                         uint64_t*& bars) {
    ring = smem + size_t(warp) * NST * QR * 4 * 256;
    bars = reinterpret_cast<uint64_t*>(smem + size_t(NW) * NST * QR * 4 * 256) + warp * NST;
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NST; ++i) mbar_init(&bars[i], 32);
        fence_mbar_init();
    }
    __syncwarp();
}

// resident blocks the inner-unit kernels of the two-quad-halo pipelines
// (CDF 9/7, CDF 5/3) are held to: one staged row loop fits the register budget
// of five 4-warp blocks per SM; the DD 13/7 pipelines (six-row rings) and the
// edge-unit kernels are left to the compiler
template <class Pipe, int CLS>
struct InvMinBlocks {
    static constexpr int value = (CLS == UNITS_INNER && PipeGeom<Pipe>::HALO == 2) ? 5 : 1;
};

// One level of one image.  UNITS_ALL: the warps take their units from Pieces;
// otherwise the units of class CLS, dealt round-robin in segment-major order.
template <class Pipe, class BT, bool ADJ, int QL, int NW, int CLS = UNITS_ALL>
__global__ void __launch_bounds__(NW * 32, InvMinBlocks<Pipe, CLS>::value) inv_kernel(const InvParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* ring;
    uint64_t* bars;
    inv_ring<INV_QR, INV_NST, NW>(smem, warp, lane, ring, bars);
    // a second launch of a level (PDL) shares no data with the first
    griddep_launch_dependents();
    uint32_t gstage = 0;
    if constexpr (CLS == UNITS_ALL) {
        Pieces<InvParams> pieces(p, blockIdx.x * NW + warp, gridDim.x * NW);
        int s, R0, R1;
        while (pieces.next(p, s, R0, R1))
            if (!inv_unit_any<Pipe, BT, ADJ, INV_QR, INV_NST>(p, s, R0, R1, lane, ring, bars, gstage)) return;
    } else {
        const int n = inv_class_units(p, CLS);
        for (int lu = blockIdx.x * NW + warp; lu < n; lu += gridDim.x * NW) {
            int s, g;
            inv_class_unit(p, CLS, lu, s, g);
            const int R0 = g * p.seg_rows;
            if (!inv_unit_any<Pipe, BT, ADJ, INV_QR, INV_NST, CLS>(p, s, R0, min(R0 + p.seg_rows, p.hq), lane, ring,
                                                                    bars, gstage))
                return;
        }
    }
}

// One level of a group of images (InvGroupLaunch): the units of class CLS of
// every image, in order, the image found by binary search over the group's
// unit ranges; only the first launch of a level waits for earlier work.
template <class Pipe, class BT, bool ADJ, int QL, int NW, int CLS = UNITS_ALL>
__global__ void __launch_bounds__(NW * 32, InvMinBlocks<Pipe, CLS>::value)
    inv_group_kernel(const __grid_constant__ InvGroupLaunch L) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* ring;
    uint64_t* bars;
    inv_ring<INV_QR, INV_NST, NW>(smem, warp, lane, ring, bars);
    if (L.wait_prev) griddep_wait();
    griddep_launch_dependents();
    uint32_t gstage = 0;
    for (int u = blockIdx.x * NW + warp; u < L.n_units[CLS]; u += gridDim.x * NW) {
        int lo = 0, hi = L.n_img - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.img[mid].u_begin[CLS] <= u) lo = mid;
            else hi = mid - 1;
        }
        const InvParams& p = L.img[lo].p;
        int s, g;
        inv_class_unit(p, CLS, u - L.img[lo].u_begin[CLS], s, g);
        const int R0 = g * p.seg_rows;
        if (!inv_unit_any<Pipe, BT, ADJ, INV_QR, INV_NST, CLS>(p, s, R0, min(R0 + p.seg_rows, p.hq), lane, ring, bars,
                                                                gstage))
            return;
    }
}

}  // namespace dwt2

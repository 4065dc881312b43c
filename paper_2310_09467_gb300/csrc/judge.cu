// judge.cu -- per-pixel prediction, the score and choice stages of the
// two-dimensional image entropy criterion, and the allocation-free judge
// (Sec. 2.1.1, Sec. 2.1.2, Eq. (1), Fig. 2a/2c).
//
// What lfc_judge and lfc_compress use from this file: the segment fixup
// (cross-CTA chain links and the bucket-boundary pairs), the fixed-point log2
// table, the entropy score sum_t P_t L2(P_t), the argmax, the copy of each
// frame's chosen candidate stream out of the judge's candidate streams, and
// the per-pixel symbol kernels for caller-given ids (emit_kernel) and for
// lfc_symbols. Candidate emission and the pair histograms of those calls run
// in judge_stream.cu.
//
// The pair counting rests on this: sorting the rotations of S by their first
// byte only, ties in generation order, puts the rotations that start with
// byte b in increasing start order, and their last bytes are the
// predecessors S[i-1] of the occurrences i of b. The last column L is the
// concatenation over b = 0..255 of those predecessor lists, so the 16-bit
// pairs of adjacent L entries are
//   (S[i-1], S[j-1]) for consecutive occurrences i < j of the same byte b,
//   (last predecessor of bucket b, first predecessor of the next non-empty
//    bucket)  -- at most 255 bucket-boundary pairs,
// with S[-1] = S[n-1].
//
// judge_hist_kernel serves only lfc_judge_noalloc (end of the file): it
// computes the symbols of its rows on the fly (no candidate stream in
// memory) and walks them in 32-byte windows, __match_any_sync finding equal
// bytes in a window and a per-warp table carrying the last predecessor of
// every byte value across windows; pairs go to a shared-memory histogram
// with warp-aggregated atomics, and per-warp / per-segment first and last
// predecessor tables stitch the chains in the fixup kernel.
#include "lfc_common.cuh"

namespace lfc {

// ------------------------------------------------------------ prediction
__device__ __forceinline__ int32_t as_i16(uint32_t v) { return (int32_t)(int16_t)(uint16_t)v; }

// Base field: raw count, or signed 16-bit difference to the previous frame.
__device__ __forceinline__ int32_t base_field(const FrameDev &F, int y, int x, bool tmp) {
    size_t k = (size_t)y * F.W + x;
    uint32_t a = __ldg(F.X + k);
    if (!tmp) return (int32_t)a;
    return as_i16(a - (uint32_t)__ldg(F.prev + k));
}

// Lossless-JPEG predictor set, floor division by arithmetic shift.
__device__ __forceinline__ int32_t jpeg_pred(int f, int32_t A, int32_t B, int32_t C) {
    switch (f) {
    case 1: return A;
    case 2: return B;
    case 3: return C;
    case 4: return A + B - C;
    case 5: return A + ((B - C) >> 1);
    case 6: return B + ((A - C) >> 1);
    case 7: return (A + B) >> 1;
    default: return 0;
    }
}

// 2-D grid rule: origin 0, first row from the left, first column from the top.
__device__ __forceinline__ int32_t grid_pred(int f, int row, int col, int32_t A, int32_t B, int32_t C) {
    if (row == 0) return col == 0 ? 0 : A;
    if (col == 0) return B;
    return jpeg_pred(f, A, B, C);
}

__device__ __forceinline__ uint32_t intra_res(const FrameDev &F, int f, int y, int x, bool tmp) {
    const int v = y % F.p, u = x % F.p;
    int32_t X = base_field(F, y, x, tmp);
    int32_t A = u > 0 ? base_field(F, y, x - 1, tmp) : 0;
    int32_t B = v > 0 ? base_field(F, y - 1, x, tmp) : 0;
    int32_t C = (u > 0 && v > 0) ? base_field(F, y - 1, x - 1, tmp) : 0;
    return (uint32_t)(X - grid_pred(f, v, u, A, B, C)) & 0xFFFFu;
}

__device__ __forceinline__ uint32_t inter_res(const FrameDev &F, int f, int y, int x, bool tmp) {
    const int t = y / F.p, s = x / F.p, p = F.p;
    int32_t X = base_field(F, y, x, tmp);
    int32_t A = s > 0 ? base_field(F, y, x - p, tmp) : 0;
    int32_t B = t > 0 ? base_field(F, y - p, x, tmp) : 0;
    int32_t C = (s > 0 && t > 0) ? base_field(F, y - p, x - p, tmp) : 0;
    return (uint32_t)(X - grid_pred(f, t, s, A, B, C)) & 0xFFFFu;
}

__device__ __forceinline__ uint32_t phase_res(const FrameDev &F, int f, int y, int x, bool tmp) {
    const int t = y / F.p, s = x / F.p, p = F.p;
    int32_t E = as_i16(intra_res(F, f, y, x, tmp));
    int32_t A = s > 0 ? as_i16(intra_res(F, f, y, x - p, tmp)) : 0;
    int32_t B = t > 0 ? as_i16(intra_res(F, f, y - p, x, tmp)) : 0;
    int32_t C = (s > 0 && t > 0) ? as_i16(intra_res(F, f, y - p, x - p, tmp)) : 0;
    return (uint32_t)(E - grid_pred(f, t, s, A, B, C)) & 0xFFFFu;
}

// Symbol of pixel (y, x) under candidate id.
__device__ __forceinline__ uint32_t pixel_symbol(const FrameDev &F, int id, int y, int x) {
    const int f = id_f(id), dom = id_dom(id);
    const bool tmp = id_tmp(id);
    uint32_t e;
    if (f == 0) {
        if (!tmp) return __ldg(F.X + (size_t)y * F.W + x);
        e = (uint32_t)base_field(F, y, x, true) & 0xFFFFu;
    } else if (dom == 0) {
        e = intra_res(F, f, y, x, tmp);
    } else if (dom == 1) {
        e = inter_res(F, f, y, x, tmp);
    } else {
        e = phase_res(F, f, y, x, tmp);
    }
    // zigzag of the residual as a signed 16-bit value
    const int32_t sv = as_i16(e);
    return (uint32_t)((sv << 1) ^ (sv >> 31)) & 0xFFFFu;
}

// Stream row r of ordering `ord` is raw row y; stream column c is raw column x.
__device__ __forceinline__ int stream_row_to_y(const FrameDev &F, int ord, int r) {
    return ord ? (r % F.Ny) * F.p + r / F.Ny : r;
}
__device__ __forceinline__ int raw_x_to_col(const FrameDev &F, int ord, int x) {
    return ord ? (x % F.p) * F.Nx + x / F.p : x;
}
__device__ __forceinline__ int col_to_raw_x(const FrameDev &F, int ord, int c) {
    return ord ? (c % F.Nx) * F.p + c / F.Nx : c;
}

// The judged byte string as rows: the (lo, hi) layout has H rows of 2W
// bytes (stream row r); the planar layout 2H rows of W bytes, rows r < H the
// high bytes of stream row r, rows H + r its low bytes.
__device__ __forceinline__ int byte_rows(const FrameDev &F, int id) { return id_planar(id) ? 2 * F.H : F.H; }

// Last byte of byte row r - 1 (the byte before the row's first byte); for
// r = 0 the string's last byte (rotation 0 wraps around).
__device__ __forceinline__ uint32_t byte_before_row(const FrameDev &F, int id, int r) {
    const int ord = id_ord(id);
    const int rr = (r == 0 ? byte_rows(F, id) : r) - 1;
    const int sr = rr % F.H;  // stream row
    const uint32_t z = pixel_symbol(F, id, stream_row_to_y(F, ord, sr), col_to_raw_x(F, ord, F.W - 1));
    const bool low = id_planar(id) && rr >= F.H;
    return low ? (z & 0xFFu) : (z >> 8);
}

// ------------------------------------------------------------ the judge
constexpr int kJudgeWarps = 16;
constexpr uint16_t kNone = 0xFFFF;

__device__ __forceinline__ int find_frame(const JudgeFrame *fr, int n, int64_t cta) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (fr[mid].cta_base <= cta) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// smem: hist[32768] u32 | first[NW][256] u16 | last[NW][256] u16 | rows[NW][maxW] u16
__global__ void __launch_bounds__(kJudgeWarps * 32, 1)
judge_hist_kernel(const JudgeFrame *__restrict__ frames, int nframes, const uint8_t *__restrict__ cand,
                  uint32_t *__restrict__ hist, uint16_t *__restrict__ summ, int maxW) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *sh_hist = reinterpret_cast<uint32_t *>(smem);
    uint16_t *sh_first = reinterpret_cast<uint16_t *>(smem + 32768 * 4);
    uint16_t *sh_last = sh_first + kJudgeWarps * 256;
    uint16_t *sh_rows = sh_last + kJudgeWarps * 256;

    const int fi = find_frame(frames, nframes, blockIdx.x);
    const JudgeFrame &J = frames[fi];
    const FrameDev F = J.F;
    const int64_t local = (int64_t)blockIdx.x - J.cta_base;
    const int ci = (int)(local / J.segs), seg = (int)(local % J.segs);
    const int id = cand[J.cand_off + ci];
    const int ord = id_ord(id);
    const bool planar = id_planar(id);
    uint32_t *ghist = hist + (size_t)(J.hist_off + ci) * kHistBins;

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r_seg0 = seg * J.rows_per_seg;
    const int r_seg1 = min(byte_rows(F, id), r_seg0 + J.rows_per_seg);
    const int rpw = (r_seg1 - r_seg0 + kJudgeWarps - 1) / kJudgeWarps;
    const int r0 = min(r_seg1, r_seg0 + w * rpw), r1 = min(r_seg1, r0 + rpw);
    uint16_t *zrow = sh_rows + (size_t)w * maxW;
    const uint8_t *zbytes = reinterpret_cast<const uint8_t *>(zrow);
    uint16_t *my_first = sh_first + w * 256, *my_last = sh_last + w * 256;
    const int nb = planar ? F.W : 2 * F.W;  // bytes per row

    uint32_t carry0 = 0;
    if (r0 < r1) carry0 = byte_before_row(F, id, r0);  // uniform per warp

    for (int pass = 0; pass < 2; pass++) {
        for (int i = threadIdx.x; i < 32768; i += blockDim.x) sh_hist[i] = 0;
        for (int i = lane; i < 256; i += 32) { my_first[i] = kNone; my_last[i] = kNone; }
        __syncthreads();
        uint32_t prev_byte = carry0;
        for (int r = r0; r < r1; r++) {
            const int sr = r % F.H;                                 // stream row of byte row r
            const int sh = planar ? (r < F.H ? 8 : 0) : 0;          // planar: the high or the low bytes
            const int y = stream_row_to_y(F, ord, sr);
            for (int x = lane; x < F.W; x += 32) zrow[raw_x_to_col(F, ord, x)] = (uint16_t)pixel_symbol(F, id, y, x);
            __syncwarp();
            auto row_byte = [&](int q) -> uint32_t { return planar ? ((uint32_t)zrow[q] >> sh) & 0xFFu : zbytes[q]; };
            for (int base = 0; base < nb; base += 32) {
                const int q = base + lane;
                const bool valid = q < nb;
                const uint32_t b = valid ? row_byte(q) : 0u;
                const uint32_t a = valid ? (q > 0 ? row_byte(q - 1) : prev_byte) : 0u;
                const uint32_t m = __match_any_sync(LFC_FULL, valid ? b : 256u + lane);
                const uint32_t lower = m & lanemask_lt();
                const int pl = lower ? 31 - __clz(lower) : lane;
                const uint32_t a_prev = __shfl_sync(LFC_FULL, a, pl);
                int bin = -1;
                if (valid) {
                    if (lower) {
                        bin = (int)((a_prev << 8) | a);
                    } else {
                        const uint16_t pend = my_last[b];
                        if (pend != kNone) bin = (int)(((uint32_t)pend << 8) | a);
                        else my_first[b] = (uint16_t)a;
                    }
                }
                __syncwarp();
                if (valid && (m & lanemask_gt()) == 0) my_last[b] = (uint16_t)a;
                __syncwarp();
                const bool contrib = bin >= 0 && (bin >> 15) == pass;
                const uint32_t hm = __match_any_sync(LFC_FULL, contrib ? (uint32_t)bin : 0x10000u + lane);
                if (contrib && (hm & lanemask_lt()) == 0) atomicAdd(&sh_hist[bin & 0x7FFF], __popc(hm));
            }
            prev_byte = row_byte(nb - 1);
            __syncwarp();
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 32768; i += blockDim.x) {
            const uint32_t c = sh_hist[i];
            if (c) atomicAdd(&ghist[pass * 32768 + i], c);
        }
        __syncthreads();
    }
    // stitch warps in stream order; write this segment's first/last tables
    if (threadIdx.x < 256) {
        const int b = threadIdx.x;
        uint16_t first = kNone, cur = kNone;
        for (int ww = 0; ww < kJudgeWarps; ww++) {
            const uint16_t f = sh_first[ww * 256 + b];
            if (f == kNone) continue;
            if (cur != kNone) atomicAdd(&ghist[((uint32_t)cur << 8) | f], 1u);
            else first = f;
            cur = sh_last[ww * 256 + b];
        }
        uint16_t *out = summ + (size_t)(J.summ_off + (int64_t)ci * J.segs + seg) * 512;
        out[b] = first;
        out[256 + b] = cur;
    }
}

// One CTA (256 threads) per (frame, candidate): links segments and adds the
// bucket-boundary pairs.
__global__ void judge_fixup_kernel(const JudgeFrame *__restrict__ frames, const int32_t *__restrict__ hist_frame,
                                   const uint8_t *__restrict__ cand, uint32_t *__restrict__ hist,
                                   const uint16_t *__restrict__ summ) {
    __shared__ uint16_t gfirst[256], glast[256];
    const int hidx = blockIdx.x;  // global histogram index
    const JudgeFrame &J = frames[hist_frame[hidx]];
    const int ci = (int)(hidx - J.hist_off);
    if (J.mask && !cand_on(J, cand[J.cand_off + ci])) return;
    uint32_t *ghist = hist + (size_t)hidx * kHistBins;
    const int b = threadIdx.x;
    uint16_t first = kNone, cur = kNone;
    for (int sgi = 0; sgi < J.segs; sgi++) {
        const uint16_t *s = summ + (size_t)(J.summ_off + (int64_t)ci * J.segs + sgi) * 512;
        const uint16_t f = s[b];
        if (f == kNone) continue;
        if (cur != kNone) atomicAdd(&ghist[((uint32_t)cur << 8) | f], 1u);
        else first = f;
        cur = s[256 + b];
    }
    gfirst[b] = first;
    glast[b] = cur;
    __syncthreads();
    if (cur != kNone) {
        for (int nb = b + 1; nb < 256; nb++) {
            if (gfirst[nb] != kNone) {
                atomicAdd(&ghist[((uint32_t)cur << 8) | gfirst[nb]], 1u);
                break;
            }
        }
    }
}

// Fixed-point 2^32 log2(c): integer part from the leading bit, 32 fraction
// bits by squaring the Q62 mantissa (128-bit product via __umul64hi).
__device__ __forceinline__ uint64_t log2_fx(uint32_t c) {
    if (c <= 1) return 0;
    const int k = 31 - __clz(c);
    uint64_t y = (uint64_t)c << (62 - k);
    uint64_t frac = 0;
#pragma unroll 4
    for (int i = 0; i < 32; i++) {
        const uint64_t hi = __umul64hi(y, y), lo = y * y;
        const uint64_t z = (hi << 2) | (lo >> 62);
        frac <<= 1;
        if (z >> 63) { frac |= 1; y = z >> 1; } else { y = z; }
    }
    return ((uint64_t)k << 32) | frac;
}

__global__ void l2_table_kernel(uint64_t *tab) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < kHistBins) tab[c] = log2_fx((uint32_t)c);
}

// One CTA per histogram: score = sum_t P_t * L2(P_t).
__global__ void __launch_bounds__(1024) entropy_kernel(const uint32_t *__restrict__ hist, const uint64_t *__restrict__ tab,
                                                       const JudgeFrame *__restrict__ frames, const int32_t *__restrict__ hist_frame,
                                                       const uint8_t *__restrict__ cand, uint64_t *__restrict__ scores,
                                                       const int32_t *__restrict__ frame_index) {
    __shared__ uint64_t part[32];
    const int hidx = blockIdx.x;
    {
        const JudgeFrame &J = frames[hist_frame[hidx]];
        if (J.mask && !cand_on(J, cand[J.cand_off + (hidx - J.hist_off)])) return;
    }
    const uint4 *h4 = reinterpret_cast<const uint4 *>(hist + (size_t)hidx * kHistBins);
    uint64_t s = 0;
    for (int i = threadIdx.x; i < kHistBins / 4; i += blockDim.x) {
        const uint4 v = h4[i];
        const uint32_t c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (c[k] > 1) s += (uint64_t)c[k] * (c[k] < (uint32_t)kHistBins ? __ldg(tab + c[k]) : log2_fx(c[k]));
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint64_t t = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0;
        t = warp_sum(t);
        if (threadIdx.x == 0) {
            const int f = hist_frame[hidx];
            const JudgeFrame &J = frames[f];
            const int id = cand[J.cand_off + (hidx - J.hist_off)];
            scores[(size_t)frame_index[f] * 256 + id] = t;
        }
    }
}

// One warp per frame: best = highest score, ties to the lowest id.
__global__ void argmax_kernel(const JudgeFrame *__restrict__ frames, int nframes, const uint8_t *__restrict__ cand,
                              const uint64_t *__restrict__ scores, uint8_t *__restrict__ choice,
                              const int32_t *__restrict__ frame_index) {
    const int f = blockIdx.x;
    if (f >= nframes) return;
    const JudgeFrame &J = frames[f];
    const uint64_t *sc = scores + (size_t)frame_index[f] * 256;
    uint64_t best = 0;
    int best_id = 256;
    for (int k = threadIdx.x; k < J.K; k += 32) {
        const int id = cand[J.cand_off + k];
        if (!cand_on(J, id)) continue;
        const uint64_t v = sc[id];
        if (best_id == 256 || v > best || (v == best && id < best_id)) { best = v; best_id = id; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t ob = __shfl_xor_sync(LFC_FULL, best, o);
        const int oi = __shfl_xor_sync(LFC_FULL, best_id, o);
        if (oi != 256 && (best_id == 256 || ob > best || (ob == best && oi < best_id))) { best = ob; best_id = oi; }
    }
    if (threadIdx.x == 0) choice[frame_index[f]] = (uint8_t)best_id;
}

cudaError_t init_l2_table(uint64_t *tab, cudaStream_t s) {
    l2_table_kernel<<<kHistBins / 256, 256, 0, s>>>(tab);
    return cudaGetLastError();
}

size_t judge_smem_bytes(int maxW) {
    return (size_t)32768 * 4 + (size_t)kJudgeWarps * 256 * 2 * 2 + (size_t)kJudgeWarps * maxW * 2;
}

cudaError_t launch_judge(lfc_plan P, const JudgeFrame *d_frames, int nframes, int64_t total_ctas,
                         const JudgeLaunch &L, const uint8_t *d_cand, int64_t nhist, uint64_t *d_scores,
                         uint8_t *d_choice) {
    cudaStream_t s = P->stream;
    Workspace &ws = P->ws;
    cudaError_t e = cudaMemsetAsync(ws.hist, 0, (size_t)nhist * kHistBins * 4, s);
    if (e != cudaSuccess) return e;
    // frame index table and hist->frame table ride behind the frame table
    const int32_t *d_frame_index = reinterpret_cast<const int32_t *>(d_frames + nframes);
    const int32_t *d_hist_frame = d_frame_index + nframes;
    stage_begin(P, LFC_STAGE_JUDGE_EMIT);
    e = launch_emit_all(P, d_frames, nframes, d_cand, L.max_tiles, L.TS, L.nslots_max, L.any_temporal, L.max_p);
    stage_end(P, LFC_STAGE_JUDGE_EMIT);
    if (e != cudaSuccess) return e;
    stage_begin(P, LFC_STAGE_JUDGE_HIST);
    e = launch_chain_hist(P, d_frames, nframes, d_cand, total_ctas, L.range_bytes);
    stage_end(P, LFC_STAGE_JUDGE_HIST);
    if (e != cudaSuccess) return e;
    stage_begin(P, LFC_STAGE_JUDGE_SCORE);
    judge_fixup_kernel<<<(unsigned)nhist, 256, 0, s>>>(d_frames, d_hist_frame, d_cand, ws.hist, ws.summ);
    entropy_kernel<<<(unsigned)nhist, 1024, 0, s>>>(ws.hist, ws.l2tab, d_frames, d_hist_frame, d_cand, d_scores,
                                                   d_frame_index);
    argmax_kernel<<<nframes, 32, 0, s>>>(d_frames, nframes, d_cand, d_scores, d_choice, d_frame_index);
    stage_end(P, LFC_STAGE_JUDGE_SCORE);
    count_launches(P, 3);
    return cudaGetLastError();
}

// ------------------------------------------------------------ emission
struct EmitArgs {
    FrameDev F[8];
    uint8_t *dst[8];
};

// Stream of the chosen id: thread per output symbol, 2-D grid (chunk, frame).
// The judge has already written every candidate's stream: copy the chosen
// one of each frame of a judge launch to the frame's stream slot (16-byte
// aligned slots; a byte tail for odd sizes).
__global__ void copy_chosen_kernel(const JudgeFrame *__restrict__ frames, int nframes, const uint8_t *__restrict__ cand,
                                   const uint8_t *__restrict__ choice, const uint8_t *__restrict__ cstream, int64_t cslot,
                                   int kmax, uint8_t *const *__restrict__ dst) {
    __shared__ int slot;
    const int i = blockIdx.y;
    const JudgeFrame &J = frames[i];
    const int g = reinterpret_cast<const int32_t *>(frames + nframes)[i];  // frame index of the call
    if (threadIdx.x == 0) {
        slot = -1;
        const int c = choice[g];
        for (int k = 0; k < J.K; k++)
            if (cand[J.cand_off + k] == c) { slot = k; break; }
    }
    __syncthreads();
    if (slot < 0) return;  // the choice is always one of the frame's candidates
    const uint8_t *src = cstream + ((size_t)i * kmax + slot) * (size_t)cslot;
    uint8_t *d = dst[g];
    const int64_t n = 2LL * J.F.W * J.F.H, n16 = n / 16;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n16; q += stride)
        reinterpret_cast<uint4 *>(d)[q] = __ldg(reinterpret_cast<const uint4 *>(src) + q);
    for (int64_t q = n16 * 16 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) d[q] = src[q];
}

cudaError_t launch_copy_chosen(lfc_plan P, const JudgeFrame *d_frames, int nframes, const uint8_t *d_cand,
                               const uint8_t *d_choice, uint8_t *const *d_dst) {
    copy_chosen_kernel<<<dim3(64, nframes), 256, 0, P->stream>>>(d_frames, nframes, d_cand, d_choice, P->ws.cstream,
                                                                  P->ws.cstream_slot, P->ws.cstream_kmax, d_dst);
    count_launches(P, 1);
    return cudaGetLastError();
}

__global__ void emit_kernel(EmitArgs args, const uint8_t *__restrict__ choice, int nframes) {
    const int f = blockIdx.y;
    if (f >= nframes) return;
    const FrameDev F = args.F[f];
    int id = choice[f];
    if ((id & 0x80) && !F.prev) id &= 0x7F;  // no reference frame: never read through NULL
    const int ord = id_ord(id);
    const bool planar = id_planar(id);
    const int64_t n = (int64_t)F.W * F.H;
    uint16_t *out = reinterpret_cast<uint16_t *>(args.dst[f]);
    uint8_t *out8 = args.dst[f];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(k / F.W), c = (int)(k % F.W);
        const int y = stream_row_to_y(F, ord, r), x = col_to_raw_x(F, ord, c);
        const uint32_t z = pixel_symbol(F, id, y, x);
        if (planar) {
            out8[k] = (uint8_t)(z >> 8);
            out8[n + k] = (uint8_t)z;
        } else {
            out[k] = (uint16_t)z;
        }
    }
}

cudaError_t launch_emit(const FrameDev *h_frames, const uint8_t *d_choice, int nframes, uint8_t *const *h_dst,
                        cudaStream_t s) {
    for (int f0 = 0; f0 < nframes; f0 += 8) {
        EmitArgs a;
        const int cnt = nframes - f0 < 8 ? nframes - f0 : 8;
        for (int i = 0; i < cnt; i++) { a.F[i] = h_frames[f0 + i]; a.dst[i] = h_dst[f0 + i]; }
        dim3 grid(1216, cnt);
        emit_kernel<<<grid, 256, 0, s>>>(a, d_choice + f0, cnt);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

__global__ void symbols_one_kernel(FrameDev F, int id, uint16_t *out) {
    const int ord = id_ord(id);
    const int64_t n = (int64_t)F.W * F.H;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(k / F.W), c = (int)(k % F.W);
        out[k] = (uint16_t)pixel_symbol(F, id, stream_row_to_y(F, ord, r), col_to_raw_x(F, ord, c));
    }
}

cudaError_t launch_symbols_one(const FrameDev &F, int id, uint16_t *dst, cudaStream_t s) {
    symbols_one_kernel<<<1216, 256, 0, s>>>(F, id, dst);
    return cudaGetLastError();
}

}  // namespace lfc

// ============================================================ no allocation
// lfc_judge_noalloc: the judge of one frame for callers that may not allocate
// device memory. It launches the kernels above one candidate at a time with
// all of their scratch in one file-scope device array, so no call allocates.
// (The paper has no counterpart; see include/lfc.h.)
namespace lfc {

constexpr int kNoAllocRowsPerSeg = 128;
constexpr int kNoAllocMaxSegs = 32;      // frames up to 32 * 128 = 4096 rows
constexpr int kNoAllocMaxWidth = 2656;   // judge_smem_bytes(2656) = 227 KB, the per-CTA limit
constexpr uint32_t kNoAllocTableMagic = 0x4C325442u;  // marks a filled log2 table

struct NoAllocScratch {
    uint32_t hist[kHistBins];                 // one candidate's pair histogram
    uint64_t l2tab[kHistBins];                // fixed-point log2 table
    uint16_t summ[kNoAllocMaxSegs * 512];     // per-segment first/last tables
    uint64_t scores[256];                     // score by id
    JudgeFrame jf_one[256];                   // candidate i: K = 1, cand_off = i
    JudgeFrame jf_all;                        // all candidates, for the argmax
    int32_t zero[4];                          // frame_index / hist_frame tables = {0}
    uint8_t cand[256];
    uint32_t table_magic;                     // kNoAllocTableMagic once l2tab holds the table
    uint32_t table_done;                      // CTAs of the filling launch that have finished
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

struct IdList {
    uint8_t id[256];
    int32_t n;
};

// Fills the log2 table unless the array already holds it. The array starts
// zeroed whenever the library's device code is loaded into a context (a new
// process, or a context re-created after a device reset), so the marker is
// then missing and the table is rebuilt; otherwise every CTA returns at once.
// The last CTA to finish sets the marker, so no CTA of a later launch can see
// the marker before the whole table is written.
__global__ void __launch_bounds__(1024) noalloc_table_kernel(NoAllocScratch *s) {
    if (*reinterpret_cast<volatile uint32_t *>(&s->table_magic) == kNoAllocTableMagic) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    s->l2tab[c] = log2_fx((uint32_t)c);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(&s->table_done, 1u) == gridDim.x - 1) {
        s->table_done = 0;
        __threadfence();
        atomicExch(&s->table_magic, kNoAllocTableMagic);
    }
}

__global__ void noalloc_describe_kernel(NoAllocScratch *s, FrameDev F, IdList ids, int segs) {
    const int i = threadIdx.x;
    if (i < ids.n) {
        s->cand[i] = ids.id[i];
        JudgeFrame &J = s->jf_one[i];
        J.F = F;
        J.K = 1;
        J.cand_off = i;
        J.segs = segs;
        J.rows_per_seg = id_planar(ids.id[i]) ? 2 * kNoAllocRowsPerSeg : kNoAllocRowsPerSeg;  // 2H rows of W bytes
        J.cta_base = 0;
        J.hist_off = 0;
        J.summ_off = 0;
        J.mask = nullptr;
    }
    if (i == 0) {
        s->jf_all = s->jf_one[0];
        s->jf_all.K = ids.n;
        s->jf_all.cand_off = 0;
        for (int k = 0; k < 4; k++) s->zero[k] = 0;
    }
}

__global__ void noalloc_copy_scores_kernel(const NoAllocScratch *s, IdList ids, uint64_t *out) {
    const int i = threadIdx.x;
    if (i < ids.n) out[ids.id[i]] = s->scores[ids.id[i]];
}

}  // namespace lfc

extern "C" int lfc_judge_noalloc(const lfc_frame *frame, const uint8_t *h_ids, int n_ids, uint8_t *d_choice,
                                 uint64_t *d_scores, void *cuda_stream) {
    using namespace lfc;
    if (!frame || !frame->data || !d_choice || !h_ids || n_ids < 1 || n_ids > 256 || frame->reserved != 0)
        return LFC_ERR_INVALID_ARG;
    const int W = frame->width, H = frame->height, p = frame->pitch;
    if (W <= 0 || H <= 0 || p <= 0 || W % p || H % p || (int64_t)W * H * 2 > ((int64_t)1 << 26))
        return LFC_ERR_INVALID_ARG;
    if (W > kNoAllocMaxWidth || H > kNoAllocMaxSegs * kNoAllocRowsPerSeg) return LFC_ERR_INVALID_ARG;
    IdList ids;
    ids.n = n_ids;
    for (int i = 0; i < n_ids; i++) {
        const int id = h_ids[i], f = id_f(id), dom = id_dom(id);
        if (dom > 2 || (f == 0 && dom != 0)) return LFC_ERR_INVALID_ARG;
        if ((id & 0x80) && !frame->prev) return LFC_ERR_INVALID_ARG;
        ids.id[i] = (uint8_t)id;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    // An error left pending by earlier work on this thread would be taken
    // for this call's own: refuse to start, and leave it in place.
    if (cudaPeekAtLastError() != cudaSuccess) return LFC_ERR_CUDA;
    // The array's device address, looked up on every call (host code may not
    // use the symbol itself, and the address changes if the context is
    // re-created).
    void *sp = nullptr;
    if (cudaGetSymbolAddress(&sp, g_noalloc_scratch) != cudaSuccess || !sp) {
        cudaGetLastError();
        return LFC_ERR_CUDA;
    }
    NoAllocScratch *s = reinterpret_cast<NoAllocScratch *>(sp);
    // One value for every call (the largest frame allowed), so that callers
    // on several host threads never set different limits.
    if (cudaFuncSetAttribute(judge_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)judge_smem_bytes(kNoAllocMaxWidth)) != cudaSuccess) {
        cudaGetLastError();
        return LFC_ERR_CUDA;
    }
    FrameDev F;
    F.X = frame->data;
    F.prev = frame->prev;
    F.W = W;
    F.H = H;
    F.p = p;
    F.Nx = W / p;
    F.Ny = H / p;
    const int segs = (H + kNoAllocRowsPerSeg - 1) / kNoAllocRowsPerSeg;
    const size_t smem = judge_smem_bytes(W);
    noalloc_table_kernel<<<kHistBins / 1024, 1024, 0, st>>>(s);
    noalloc_describe_kernel<<<1, 256, 0, st>>>(s, F, ids, segs);
    if (cudaGetLastError() != cudaSuccess) return LFC_ERR_CUDA;
    for (int i = 0; i < n_ids; i++) {
        if (cudaMemsetAsync(s->hist, 0, sizeof(s->hist), st) != cudaSuccess) {
            cudaGetLastError();
            return LFC_ERR_CUDA;
        }
        judge_hist_kernel<<<segs, kJudgeWarps * 32, smem, st>>>(&s->jf_one[i], 1, s->cand, s->hist, s->summ, W);
        judge_fixup_kernel<<<1, 256, 0, st>>>(&s->jf_one[i], s->zero, s->cand, s->hist, s->summ);
        entropy_kernel<<<1, 1024, 0, st>>>(s->hist, s->l2tab, &s->jf_one[i], s->zero, s->cand, s->scores, s->zero);
        if (cudaGetLastError() != cudaSuccess) return LFC_ERR_CUDA;
    }
    argmax_kernel<<<1, 32, 0, st>>>(&s->jf_all, 1, s->cand, s->scores, d_choice, s->zero);
    if (d_scores) noalloc_copy_scores_kernel<<<1, 256, 0, st>>>(s, ids, d_scores);
    return cudaGetLastError() == cudaSuccess ? LFC_OK : LFC_ERR_CUDA;
}

// judge_stream.cu -- the entropy criterion in two streaming kernels
// (Sec. 2.1.1 prediction, Sec. 2.1.2 / Eq. (1) judge).
//
// 1. emit_all_kernel: every candidate stream of a frame is written once.
//    One CTA per (lenslet row t, 16 lenslets s0.., base field kind): the
//    frame tile of lenslet rows t-1..t and lenslet columns s0-1..s0+15
//    (one lenslet of halo above and to the left) is staged in shared memory
//    as the base field (raw counts, or the signed difference to the previous
//    frame); the intra residual fields e1_f of the predictor functions in use
//    are formed once in shared memory; then every pixel's symbol is produced
//    for every candidate of the kind and stored in the candidate's ordering
//    (raw order: 480-byte row runs; view-major order: 32-byte runs).
// 2. chain_hist_kernel: one CTA per segment of a candidate stream, one
//    thread per range (2-8 KB, tuned) walking it byte by byte (see below); the
//    ranges are stitched per CTA and the CTAs by the fixup kernel.
#include "lfc_common.cuh"

namespace lfc {

// ------------------------------------------------------------- emission
constexpr int kEmitThreads = 256;

__device__ __forceinline__ int32_t jf_pred(int f, int32_t A, int32_t B, int32_t C) {
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
__device__ __forceinline__ int32_t g_pred(int f, int row, int col, int32_t A, int32_t B, int32_t C) {
    if (row == 0) return col == 0 ? 0 : A;
    if (col == 0) return B;
    return jf_pred(f, A, B, C);
}
__device__ __forceinline__ uint16_t zz16(int32_t e) {
    const int32_t s = (int32_t)(int16_t)(uint16_t)(uint32_t)e;
    return (uint16_t)(((s << 1) ^ (s >> 31)) & 0xFFFF);
}

size_t emit_all_smem_bytes(int p, int ts, int nslots) {
    const size_t cells = (size_t)(2 * p) * (size_t)((ts + 1) * p);
    return cells * 2 * (size_t)(1 + nslots) + 256;
}

// grid (tiles, frames, kind); kind 0 = raw base field, 1 = temporal difference
__global__ void __launch_bounds__(kEmitThreads) emit_all_kernel(const JudgeFrame *__restrict__ frames,
                                                                const uint8_t *__restrict__ cand, uint8_t *__restrict__ cstream,
                                                                int64_t cslot, int kmax, int TS) {
    extern __shared__ __align__(16) uint8_t esm[];
    __shared__ int16_t slot_of[8][3][2];  // candidate index for (f, domain, ordering), -1 if absent
    __shared__ int8_t eslot_of[8];        // intra residual field of f
    __shared__ uint32_t fmask_ord[2];     // f values with any candidate in that ordering
    const int fi = blockIdx.y, kind = blockIdx.z;
    const JudgeFrame &J = frames[fi];
    const FrameDev F = J.F;
    if (kind == 1 && F.prev == nullptr) return;
    const int p = F.p, Nx = F.Nx, Ny = F.Ny, W = F.W;
    const int tiles_s = (Nx + TS - 1) / TS;
    if ((int)blockIdx.x >= Ny * tiles_s) return;
    const int t = blockIdx.x / tiles_s, s0 = (blockIdx.x % tiles_s) * TS, ns = min(TS, Nx - s0);
    const int TR = 2 * p, TC = (TS + 1) * p, ncols = (ns + 1) * p;
    const int cells = TR * TC;
    uint16_t *Fb = reinterpret_cast<uint16_t *>(esm);
    int16_t *E = reinterpret_cast<int16_t *>(esm) + cells;
    uint32_t fset = 0;
    int nc = 0;
    for (int k = 0; k < J.K; k++) {
        const int id = cand[J.cand_off + k];
        if (((id >> 7) & 1) != kind || !cand_on(J, id)) continue;
        nc++;
        const int f = id & 15, dom = (id >> 4) & 3;
        if (f && dom != 1) fset |= 1u << f;
    }
    if (nc == 0) return;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 48; i++) (&slot_of[0][0][0])[i] = -1;
        fmask_ord[0] = fmask_ord[1] = 0;
        for (int f = 0; f < 8; f++) eslot_of[f] = (int8_t)__popc(fset & ((1u << f) - 1u));
        for (int k = 0; k < J.K; k++) {
            const int id = cand[J.cand_off + k];
            if (((id >> 7) & 1) != kind || !cand_on(J, id)) continue;
            const int f = id & 15, dom = (id >> 4) & 3, ord = (id >> 6) & 1;
            slot_of[f][dom][ord] = (int16_t)k;
            fmask_ord[ord] |= 1u << f;
        }
    }
    const int y0 = (t - 1) * p, x0 = (s0 - 1) * p;
    for (int q = threadIdx.x; q < TR * ncols; q += blockDim.x) {
        const int ly = q / ncols, lx = q - ly * ncols;
        const int y = y0 + ly, x = x0 + lx;
        uint32_t v = 0;
        if (y >= 0 && x >= 0) {
            const size_t k = (size_t)y * W + x;
            v = __ldg(F.X + k);
            if (kind) v = (v - (uint32_t)__ldg(F.prev + k)) & 0xFFFFu;
        }
        Fb[ly * TC + lx] = (uint16_t)v;
    }
    __syncthreads();
#define FVAL(idx) (kind ? (int32_t)(int16_t)Fb[idx] : (int32_t)Fb[idx])
    // intra residual fields (signed 16-bit) for every f in use
    for (int q = threadIdx.x; q < TR * ncols; q += blockDim.x) {
        const int ly = q / ncols, lx = q - ly * ncols;
        const int v = ly % p, u = lx % p;
        const int idx = ly * TC + lx;
        const int32_t Xv = FVAL(idx);
        const int32_t A = u > 0 ? FVAL(idx - 1) : 0;
        const int32_t B = v > 0 ? FVAL(idx - TC) : 0;
        const int32_t C = (u > 0 && v > 0) ? FVAL(idx - TC - 1) : 0;
#pragma unroll
        for (int f = 1; f < 8; f++)
            if (fset & (1u << f)) E[(size_t)eslot_of[f] * cells + idx] = (int16_t)(Xv - g_pred(f, v, u, A, B, C));
    }
    __syncthreads();
    const int n_cols_out = ns * p;
    uint16_t *base = reinterpret_cast<uint16_t *>(cstream + (size_t)fi * kmax * (size_t)cslot);
    const size_t cslot16 = (size_t)cslot / 2;
    for (int ord = 0; ord < 2; ord++) {
        const uint32_t fm = fmask_ord[ord];
        if (!fm || (int)threadIdx.x >= n_cols_out) continue;
        int lx, s;
        int64_t pos0, pstep;
        if (ord == 0) {  // thread = raw column; rows r -> raw rows t*p + r
            const int lc = threadIdx.x;
            lx = p + lc;
            s = s0 + lc / p;
            pos0 = (int64_t)(t * p) * W + (int64_t)s0 * p + lc;
            pstep = W;
        } else {         // thread = (u, lenslet); rows r -> view rows (v = r) * Ny + t
            const int u = threadIdx.x / ns, si = threadIdx.x - u * ns;
            lx = p + si * p + u;
            s = s0 + si;
            pos0 = (int64_t)t * W + (int64_t)u * Nx + s0 + si;
            pstep = (int64_t)Ny * W;
        }
        for (int r = 0; r < p; r++) {
            const int idx = (p + r) * TC + lx;
            const int64_t pos = pos0 + r * pstep;
            const int32_t Xv = FVAL(idx);
            if (fm & 1u) {
                const int k = slot_of[0][0][ord];
                base[(size_t)k * cslot16 + pos] = kind ? zz16(Xv) : (uint16_t)Xv;
            }
            const int32_t XA = s > 0 ? FVAL(idx - p) : 0;
            const int32_t XB = t > 0 ? FVAL(idx - p * TC) : 0;
            const int32_t XC = (s > 0 && t > 0) ? FVAL(idx - p * TC - p) : 0;
#pragma unroll
            for (int f = 1; f < 8; f++) {
                if (!(fm & (1u << f))) continue;
                const int k0 = slot_of[f][0][ord], k1 = slot_of[f][1][ord], k2 = slot_of[f][2][ord];
                if (k1 >= 0) base[(size_t)k1 * cslot16 + pos] = zz16(Xv - g_pred(f, t, s, XA, XB, XC));
                if (k0 >= 0 || k2 >= 0) {
                    const int16_t *Ef = E + (size_t)eslot_of[f] * cells;
                    const int32_t e = Ef[idx];
                    if (k0 >= 0) base[(size_t)k0 * cslot16 + pos] = zz16(e);
                    if (k2 >= 0) {
                        const int32_t eA = s > 0 ? Ef[idx - p] : 0;
                        const int32_t eB = t > 0 ? Ef[idx - p * TC] : 0;
                        const int32_t eC = (s > 0 && t > 0) ? Ef[idx - p * TC - p] : 0;
                        base[(size_t)k2 * cslot16 + pos] = zz16(e - g_pred(f, t, s, eA, eB, eC));
                    }
                }
            }
        }
    }
#undef FVAL
}

// ------------------------------------------------------ pair-chain histogram
// One thread walks a contiguous byte range of a candidate stream in one
// pass. Its pending table (predecessor of the last occurrence of each byte
// value, 0xFFFF before the first) holds 16-bit entries in shared memory, entry
// b of thread t in half (b % 2) of word (b / 2) * T + t, so each lane always
// hits its own bank. The first occurrence of every value in the range goes
// to a global scratch table, so the CTA can stitch the ranges in order
// afterwards. Pairs (x, y) with x, y < 64 (the hot corner for small residuals)
// are counted in shared memory, the very common pair (0, 0) in a register,
// all others with fire-and-forget atomics into the L2-resident histogram.
constexpr int kChainThreads = 384;
constexpr int kHot = 64;                                            // hot corner side
constexpr uint16_t kNoPred = 0xFFFF;

size_t chain_smem_bytes() { return (size_t)kHot * kHot * 4 + (size_t)128 * kChainThreads * 4; }
int chain_threads() { return kChainThreads; }
int64_t chain_first_bytes_per_cta() { return (int64_t)kChainThreads * 256; }

__device__ __forceinline__ int find_frame_s(const JudgeFrame *fr, int n, int64_t cta) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fr[mid].cta_base <= cta) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// tbl is indexed as word (b / 2) * T + t: callers pass the thread's column t.
__device__ __forceinline__ void chain_byte(uint32_t b, uint32_t &prev, uint32_t *tbl, int t, uint32_t *hot,
                                           uint32_t *ghist, uint8_t *first, uint32_t &c0) {
    const uint32_t a = prev;
    prev = b;
    const uint32_t wi = (b >> 1) * kChainThreads + (uint32_t)t;
    const uint32_t word = tbl[wi];
    const uint32_t sh = (b & 1u) << 4;
    const uint32_t pend = (word >> sh) & 0xFFFFu;
    if (pend != kNoPred) {
        const uint32_t both = pend | a;
        if (both == 0) {
            c0++;
        } else if (both < (uint32_t)kHot) {
            atomicAdd(&hot[pend * kHot + a], 1u);
        } else {
            atomicAdd(&ghist[(pend << 8) | a], 1u);
        }
    } else {
        first[b] = (uint8_t)a;
    }
    tbl[wi] = (word & ~(0xFFFFu << sh)) | (a << sh);
}

__device__ __forceinline__ void chain_word(uint32_t w, uint32_t &prev, uint32_t *tbl, int t, uint32_t *hot,
                                           uint32_t *ghist, uint8_t *first, uint32_t &c0) {
#pragma unroll
    for (int q = 0; q < 4; q++) chain_byte((w >> (8 * q)) & 0xFFu, prev, tbl, t, hot, ghist, first, c0);
}

__global__ void __launch_bounds__(kChainThreads)
chain_hist_kernel(const JudgeFrame *__restrict__ frames, int nframes, const uint8_t *__restrict__ cand,
                  const uint8_t *__restrict__ cstream, int64_t cslot, int kmax, uint32_t *__restrict__ hist,
                  uint16_t *__restrict__ summ, uint8_t *__restrict__ first_all, int range_bytes) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *hot = reinterpret_cast<uint32_t *>(smem);   // [kHot][kHot]
    uint32_t *tbl = hot + kHot * kHot;                    // [128][T]
    const int fi = find_frame_s(frames, nframes, blockIdx.x);
    const JudgeFrame &J = frames[fi];
    const int64_t local = (int64_t)blockIdx.x - J.cta_base;
    const int ci = (int)(local / J.segs), seg = (int)(local % J.segs);
    const uint8_t *S = cstream + ((size_t)fi * kmax + ci) * (size_t)cslot;
    uint32_t *ghist = hist + (size_t)(J.hist_off + ci) * kHistBins;
    const int64_t n = 2LL * J.F.W * J.F.H;
    const int t = threadIdx.x;
    if (!cand_on(J, cand[J.cand_off + ci])) return;  // not proposed: no stream, no histogram
    const int64_t seg_bytes = (int64_t)kChainThreads * range_bytes;
    const int64_t ra64 = min(n, (int64_t)seg * seg_bytes + (int64_t)t * range_bytes);
    const int len = (int)(min(n, ra64 + range_bytes) - ra64);
    const uint8_t *R = S + ra64;
    uint8_t *first = first_all + ((size_t)blockIdx.x * kChainThreads + t) * 256;
    for (int i = t; i < kHot * kHot; i += kChainThreads) hot[i] = 0;
    for (int k = 0; k < 128; k++) tbl[k * kChainThreads + t] = 0xFFFFFFFFu;
    __syncthreads();
    uint32_t prev = len > 0 ? (uint32_t)S[ra64 == 0 ? n - 1 : ra64 - 1] : 0u;
    uint32_t c0 = 0;
    const int full = len & ~15;
    const uint4 *R4 = reinterpret_cast<const uint4 *>(R);
    // two 16-byte loads in flight ahead of the bytes being walked
    uint4 v0 = full > 0 ? __ldg(R4) : make_uint4(0, 0, 0, 0);
    uint4 v1 = full > 16 ? __ldg(R4 + 1) : make_uint4(0, 0, 0, 0);
    for (int i0 = 0; i0 < full; i0 += 16) {
        const uint4 v2 = (i0 + 32 < full) ? __ldg(R4 + (i0 >> 4) + 2) : make_uint4(0, 0, 0, 0);
        chain_word(v0.x, prev, tbl, t, hot, ghist, first, c0);
        chain_word(v0.y, prev, tbl, t, hot, ghist, first, c0);
        chain_word(v0.z, prev, tbl, t, hot, ghist, first, c0);
        chain_word(v0.w, prev, tbl, t, hot, ghist, first, c0);
        v0 = v1;
        v1 = v2;
    }
    for (int i = full; i < len; i++) chain_byte(R[i], prev, tbl, t, hot, ghist, first, c0);
    if (c0) atomicAdd(&hot[0], c0);
    __syncthreads();
    for (int i = t; i < kHot * kHot; i += kChainThreads) {
        const uint32_t c = hot[i];
        if (c) atomicAdd(&ghist[((uint32_t)(i / kHot) << 8) | (uint32_t)(i % kHot)], c);
    }
    // stitch the threads' ranges in order (thread b handles byte value b)
    if (t < 256) {
        const int bv = t;
        const uint8_t *first_cta = first_all + (size_t)blockIdx.x * kChainThreads * 256;
        uint16_t f0 = kNoPred, cur = kNoPred;
        for (int tt = 0; tt < kChainThreads; tt++) {
            const uint16_t last = (uint16_t)((tbl[(bv >> 1) * kChainThreads + tt] >> ((bv & 1) * 16)) & 0xFFFFu);
            if (last == kNoPred) continue;
            const uint16_t f = first_cta[(size_t)tt * 256 + bv];
            if (cur != kNoPred) atomicAdd(&ghist[((uint32_t)cur << 8) | f], 1u);
            else f0 = f;
            cur = last;
        }
        uint16_t *out = summ + (size_t)(J.summ_off + (int64_t)ci * J.segs + seg) * 512;
        out[bv] = f0;
        out[256 + bv] = cur;
    }
}

cudaError_t launch_emit_all(lfc_plan P, const JudgeFrame *d_frames, int nframes, const uint8_t *d_cand, int max_tiles,
                            int TS, int nslots_max, int any_temporal, int max_p) {
    const size_t smem = emit_all_smem_bytes(max_p, TS, nslots_max);
    cudaError_t e = cudaFuncSetAttribute(emit_all_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(max_tiles, nframes, any_temporal ? 2 : 1);
    emit_all_kernel<<<grid, kEmitThreads, smem, P->stream>>>(d_frames, d_cand, P->ws.cstream, P->ws.cstream_slot,
                                                             P->ws.cstream_kmax, TS);
    count_launches(P, 1);
    return cudaGetLastError();
}

cudaError_t launch_chain_hist(lfc_plan P, const JudgeFrame *d_frames, int nframes, const uint8_t *d_cand, int64_t total_ctas,
                              int range_bytes) {
    const size_t smem = chain_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(chain_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    chain_hist_kernel<<<(unsigned)total_ctas, kChainThreads, smem, P->stream>>>(
        d_frames, nframes, d_cand, P->ws.cstream, P->ws.cstream_slot, P->ws.cstream_kmax, P->ws.hist, P->ws.summ,
        P->ws.chain_first, range_bytes);
    count_launches(P, 1);
    return cudaGetLastError();
}

}  // namespace lfc

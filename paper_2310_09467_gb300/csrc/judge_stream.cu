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
// 2. chain_hist_kernel: one CTA per 512 KB segment of a candidate stream.
//    Each warp walks its contiguous bytes in 32-byte windows staged through
//    shared memory; __match_any_sync finds equal bytes, the predecessor of
//    the previous occurrence comes by shuffle or from a per-warp pending
//    table, and pairs are counted in a shared-memory histogram of half the
//    65536 bins per pass with warp-aggregated atomics. Per-warp first/last
//    predecessor tables are stitched per CTA and across CTAs by the fixup.
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

struct CandInfo {
    uint8_t ci, f, dom, ord, slot;  // slot: e1 field index of f
};

size_t emit_all_smem_bytes(int p, int ts, int nslots) {
    const size_t cells = (size_t)(2 * p) * (size_t)((ts + 1) * p);
    return cells * 2 * (size_t)(1 + nslots) + 64 * sizeof(CandInfo) + 64;
}

// grid (tiles, frames, kind); kind 0 = raw base field, 1 = temporal difference
__global__ void __launch_bounds__(kEmitThreads) emit_all_kernel(const JudgeFrame *__restrict__ frames,
                                                                const uint8_t *__restrict__ cand, uint8_t *__restrict__ cstream,
                                                                int64_t cslot, int kmax, int TS) {
    extern __shared__ __align__(16) uint8_t esm[];
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
    // candidate list of this kind, f-set of the intra residual fields
    uint32_t fset = 0;
    int nc = 0;
    for (int k = 0; k < J.K; k++) {
        const int id = cand[J.cand_off + k];
        if (((id >> 7) & 1) != kind) continue;
        nc++;
        const int f = id & 15, dom = (id >> 4) & 3;
        if (f && dom != 1) fset |= 1u << f;
    }
    if (nc == 0) return;
    const int nslots = __popc(fset);
    CandInfo *ci_list = reinterpret_cast<CandInfo *>(E + (size_t)nslots * cells);
    if (threadIdx.x == 0) {
        int j = 0;
        for (int k = 0; k < J.K; k++) {
            const int id = cand[J.cand_off + k];
            if (((id >> 7) & 1) != kind) continue;
            CandInfo c;
            c.ci = (uint8_t)k;
            c.f = (uint8_t)(id & 15);
            c.dom = (uint8_t)((id >> 4) & 3);
            c.ord = (uint8_t)((id >> 6) & 1);
            c.slot = (uint8_t)__popc(fset & ((1u << c.f) - 1u));
            ci_list[j++] = c;
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
    // intra residual fields (signed 16-bit) for every f in use
#define FVAL(idx) (kind ? (int32_t)(int16_t)Fb[idx] : (int32_t)Fb[idx])
    for (int q = threadIdx.x; q < TR * ncols; q += blockDim.x) {
        const int ly = q / ncols, lx = q - ly * ncols;
        const int v = ly % p, u = lx % p;
        const int idx = ly * TC + lx;
        const int32_t Xv = FVAL(idx);
        const int32_t A = u > 0 ? FVAL(idx - 1) : 0;
        const int32_t B = v > 0 ? FVAL(idx - TC) : 0;
        const int32_t C = (u > 0 && v > 0) ? FVAL(idx - TC - 1) : 0;
        uint32_t fs = fset;
        int slot = 0;
        while (fs) {
            const int f = __ffs(fs) - 1;
            fs &= fs - 1;
            E[(size_t)slot * cells + idx] = (int16_t)(Xv - g_pred(f, v, u, A, B, C));
            slot++;
        }
    }
    __syncthreads();
    const int npx = p * ns * p;
    const int64_t n_sym = (int64_t)W * F.H;
    for (int ord = 0; ord < 2; ord++) {
        for (int q = threadIdx.x; q < npx; q += blockDim.x) {
            int ly, lx;
            int64_t pos;
            if (ord == 0) {
                const int lr = q / (ns * p), lc = q - lr * (ns * p);
                ly = p + lr;
                lx = p + lc;
                pos = (int64_t)(t * p + lr) * W + (int64_t)s0 * p + lc;
            } else {
                const int v = q / (p * ns), rem = q - v * (p * ns), u = rem / ns, si = rem - u * ns;
                ly = p + v;
                lx = p + si * p + u;
                pos = (int64_t)(v * Ny + t) * W + (int64_t)u * Nx + s0 + si;
            }
            const int s = s0 + (lx - p) / p;
            const int idx = ly * TC + lx;
            for (int k = 0; k < nc; k++) {
                const CandInfo c = ci_list[k];
                if (c.ord != ord) continue;
                uint16_t z;
                if (c.f == 0) {
                    z = kind ? zz16(FVAL(idx)) : Fb[idx];
                } else if (c.dom == 0) {
                    z = zz16(E[(size_t)c.slot * cells + idx]);
                } else if (c.dom == 1) {
                    const int32_t Xv = FVAL(idx);
                    const int32_t A = s > 0 ? FVAL(idx - p) : 0;
                    const int32_t B = t > 0 ? FVAL(idx - p * TC) : 0;
                    const int32_t C = (s > 0 && t > 0) ? FVAL(idx - p * TC - p) : 0;
                    z = zz16(Xv - g_pred(c.f, t, s, A, B, C));
                } else {
                    const int16_t *Ef = E + (size_t)c.slot * cells;
                    const int32_t Xv = Ef[idx];
                    const int32_t A = s > 0 ? Ef[idx - p] : 0;
                    const int32_t B = t > 0 ? Ef[idx - p * TC] : 0;
                    const int32_t C = (s > 0 && t > 0) ? Ef[idx - p * TC - p] : 0;
                    z = zz16(Xv - g_pred(c.f, t, s, A, B, C));
                }
                uint16_t *out = reinterpret_cast<uint16_t *>(cstream + ((size_t)fi * kmax + c.ci) * (size_t)cslot);
                if (pos < n_sym) out[pos] = z;
            }
        }
    }
#undef FVAL
}

// ------------------------------------------------------ pair-chain histogram
constexpr int kChainWarps = 32;
constexpr int kChunk = 512;
constexpr int64_t kSegBytes = 512 * 1024;
constexpr uint16_t kNoPred = 0xFFFF;

size_t chain_smem_bytes() { return 131072 + (size_t)kChainWarps * 256 * 2 * 2 + (size_t)kChainWarps * kChunk; }
int64_t chain_seg_bytes() { return kSegBytes; }

__device__ __forceinline__ int find_frame_s(const JudgeFrame *fr, int n, int64_t cta) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fr[mid].cta_base <= cta) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kChainWarps * 32, 1)
chain_hist_kernel(const JudgeFrame *__restrict__ frames, int nframes, const uint8_t *__restrict__ cstream, int64_t cslot,
                  int kmax, uint32_t *__restrict__ hist, uint16_t *__restrict__ summ) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *sh_hist = reinterpret_cast<uint32_t *>(smem);
    uint16_t *sh_first = reinterpret_cast<uint16_t *>(smem + 131072);
    uint16_t *sh_last = sh_first + kChainWarps * 256;
    uint8_t *sh_buf = reinterpret_cast<uint8_t *>(sh_last + kChainWarps * 256);
    const int fi = find_frame_s(frames, nframes, blockIdx.x);
    const JudgeFrame &J = frames[fi];
    const int64_t local = (int64_t)blockIdx.x - J.cta_base;
    const int ci = (int)(local / J.segs), seg = (int)(local % J.segs);
    const uint8_t *S = cstream + ((size_t)fi * kmax + ci) * (size_t)cslot;
    uint32_t *ghist = hist + (size_t)(J.hist_off + ci) * kHistBins;
    const int64_t n = 2LL * J.F.W * J.F.H;
    const int64_t a = (int64_t)seg * kSegBytes, b = min(n, a + kSegBytes);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t per = (((b - a) + kChainWarps - 1) / kChainWarps + kChunk - 1) / kChunk * kChunk;
    const int64_t wa = min(b, a + w * per), we = min(b, wa + per);
    uint16_t *my_first = sh_first + w * 256, *my_last = sh_last + w * 256;
    uint8_t *buf = sh_buf + w * kChunk;
    const uint32_t carry0 = wa < we ? (uint32_t)S[wa == 0 ? n - 1 : wa - 1] : 0u;

    for (int pass = 0; pass < 2; pass++) {
        for (int i = threadIdx.x; i < 32768; i += blockDim.x) sh_hist[i] = 0;
        for (int i = lane; i < 256; i += 32) { my_first[i] = kNoPred; my_last[i] = kNoPred; }
        __syncthreads();
        uint32_t prev = carry0;
        for (int64_t c0 = wa; c0 < we; c0 += kChunk) {
            const int cnt = (int)min((int64_t)kChunk, we - c0);
            const int64_t o = c0 + 16 * lane;
            if (o + 16 <= we) {
                *reinterpret_cast<uint4 *>(buf + 16 * lane) = __ldg(reinterpret_cast<const uint4 *>(S + o));
            } else {
                for (int k = 0; k < 16; k++) buf[16 * lane + k] = (o + k < we) ? S[o + k] : 0;
            }
            __syncwarp();
            for (int w0 = 0; w0 < cnt; w0 += 32) {
                const int q = w0 + lane;
                const bool valid = q < cnt;
                const uint32_t bb = buf[q];
                uint32_t aa = __shfl_up_sync(LFC_FULL, bb, 1);
                if (lane == 0) aa = prev;
                prev = __shfl_sync(LFC_FULL, bb, 31);
                const uint32_t m = __match_any_sync(LFC_FULL, valid ? bb : 256u + lane);
                const uint32_t lower = m & lanemask_lt();
                const int pl = lower ? 31 - __clz(lower) : lane;
                const uint32_t a_prev = __shfl_sync(LFC_FULL, aa, pl);
                int bin = -1;
                if (valid) {
                    if (lower) {
                        bin = (int)((a_prev << 8) | aa);
                    } else {
                        const uint16_t pend = my_last[bb];
                        if (pend != kNoPred) bin = (int)(((uint32_t)pend << 8) | aa);
                        else my_first[bb] = (uint16_t)aa;
                    }
                }
                __syncwarp();
                if (valid && (m & lanemask_gt()) == 0) my_last[bb] = (uint16_t)aa;
                __syncwarp();
                const bool contrib = bin >= 0 && (bin >> 15) == pass;
                const uint32_t hm = __match_any_sync(LFC_FULL, contrib ? (uint32_t)bin : 0x10000u + lane);
                if (contrib && (hm & lanemask_lt()) == 0) atomicAdd(&sh_hist[bin & 0x7FFF], (uint32_t)__popc(hm));
            }
            __syncwarp();
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 32768; i += blockDim.x) {
            const uint32_t c = sh_hist[i];
            if (c) atomicAdd(&ghist[pass * 32768 + i], c);
        }
        __syncthreads();
    }
    if (threadIdx.x < 256) {
        const int bv = threadIdx.x;
        uint16_t first = kNoPred, cur = kNoPred;
        for (int ww = 0; ww < kChainWarps; ww++) {
            const uint16_t f = sh_first[ww * 256 + bv];
            if (f == kNoPred) continue;
            if (cur != kNoPred) atomicAdd(&ghist[((uint32_t)cur << 8) | f], 1u);
            else first = f;
            cur = sh_last[ww * 256 + bv];
        }
        uint16_t *out = summ + (size_t)(J.summ_off + (int64_t)ci * J.segs + seg) * 512;
        out[bv] = first;
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

cudaError_t launch_chain_hist(lfc_plan P, const JudgeFrame *d_frames, int nframes, const uint8_t *d_cand, int64_t total_ctas) {
    (void)d_cand;
    const size_t smem = chain_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(chain_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    chain_hist_kernel<<<(unsigned)total_ctas, kChainWarps * 32, smem, P->stream>>>(
        d_frames, nframes, P->ws.cstream, P->ws.cstream_slot, P->ws.cstream_kmax, P->ws.hist, P->ws.summ);
    count_launches(P, 1);
    return cudaGetLastError();
}

}  // namespace lfc

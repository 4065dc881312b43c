// mtf_huff.cu -- move-to-front, zero-run coding, Huffman table choice and bit
// packing of every bzip2 block (Sec. 2.1.3; public bzip2 block format).
//
// MTF is sequential per block, so each block's BWT output is cut into
// 4096-byte segments handled by one warp each. A segment's effect on the MTF
// list is "its distinct symbols by most recent use, then the old list
// without them"; one warp per block composes these summaries in order to get
// every segment's starting list, then every segment replays MTF from its
// list with the 256-entry list held in registers (8 entries per lane).
#include <climits>

#include "lfc_common.cuh"

namespace lfc {

constexpr int kSymStride = kBlockCap + 64;  // uint16 symbols per block slot

// Sequence index of byte c among the bytes in use (ascending byte order).
__device__ __forceinline__ void build_seq_table(const uint32_t *in_use, uint8_t *seq) {
    for (int c = threadIdx.x; c < 256; c += blockDim.x) {
        int cnt = 0;
        const int w = c >> 5;
        for (int i = 0; i < w; i++) cnt += __popc(in_use[i]);
        cnt += __popc(in_use[w] & ((1u << (c & 31)) - 1u));
        seq[c] = (uint8_t)cnt;
    }
}

// ---------------------------------------------------- MTF: segment summaries
// The summaries (distinct bytes of each 4096-byte segment of L by last use,
// latest first) come from the BWT output kernel, as byte values.
// One CTA per block: starting list of every segment, one list entry per
// thread. Composing a segment's summary: its record first, then the old
// list without the record's symbols (kept entries compacted by a scan).
__global__ void __launch_bounds__(256) mtf_compose_kernel(const BlockState *__restrict__ st, const uint8_t *__restrict__ rec_all,
                                                          const int32_t *__restrict__ reclen_all, uint8_t *__restrict__ lists_all) {
    __shared__ uint8_t lst[256];
    __shared__ uint8_t inr[256];
    __shared__ uint8_t seq[256];
    __shared__ uint32_t iush[8];
    __shared__ int32_t rl_s[kTilesPerBlock];
    __shared__ int sh[33];
    const int b = blockIdx.x, t = threadIdx.x;
    const int m = st[b].m;
    if (t < 8) iush[t] = st[b].in_use[t];
    __syncthreads();
    build_seq_table(iush, seq);  // records hold byte values; lists hold their indices
    int n_in_use = 0;
    for (int i = 0; i < 8; i++) n_in_use += __popc(iush[i]);
    const int ng = (m + kTile - 1) / kTile;
    for (int g = t; g < ng; g += 256) rl_s[g] = reclen_all[(size_t)b * kTilesPerBlock + g];
    lst[t] = t < n_in_use ? (uint8_t)t : (uint8_t)0xFF;
    const uint8_t *recb = rec_all + (size_t)b * kTilesPerBlock * 256;
    uint8_t r_next = ng > 0 ? recb[t] : 0;
    __syncthreads();
    r_next = seq[r_next];
    for (int g = 0; g < ng; g++) {
        lists_all[((size_t)b * kTilesPerBlock + g) * 256 + t] = lst[t];
        const int rl = rl_s[g];
        const uint8_t r = r_next;
        if (g + 1 < ng) r_next = seq[recb[(size_t)(g + 1) * 256 + t]];
        inr[t] = 0;
        __syncthreads();
        if (t < rl) inr[r] = 1;
        __syncthreads();
        const uint8_t x = lst[t];
        const bool keep = t < n_in_use && !inr[x];
        const int pos = rl + block_excl_sum<int>(keep ? 1 : 0, sh, nullptr);  // syncs: all of lst is read
        if (keep) lst[pos] = x;
        if (t < rl) lst[t] = r;
        __syncthreads();
    }
}

// One warp per segment: MTF indices from the segment's starting list, 32
// positions per step. With the list (lst) and its inverse (posof) in shared
// memory at the window start, lane k with symbol s:
//  - s also at an earlier lane j of the window (the latest such j): s was at
//    the front after j and each lane i in (j, k) pushed it back one place iff
//    i's symbol was not moved to the front after j, i.e. prev(i) <= j, where
//    prev(i) is the latest earlier lane with i's symbol (-1 if none);
//  - otherwise: s is still in the old part of the list, behind the distinct
//    symbols of lanes < k, so its index is P + #{first-occurrence lanes
//    i < k with P_i > P}, P = posof[s].
// Both counts compare one value per lane with every other lane's: done
// bit-sliced over ballots of the values' bits. The list then becomes the
// window's symbols by last use, then the old list without them; entries
// behind the deepest window symbol keep their places.
__global__ void __launch_bounds__(32) mtf_encode_kernel(const BlockState *__restrict__ st, const uint8_t *__restrict__ L_all,
                                                        const uint8_t *__restrict__ lists_all, uint8_t *__restrict__ idx_all) {
    __shared__ uint8_t seq[256];
    __shared__ uint32_t iush[8];
    __shared__ uint8_t lst[256];
    __shared__ uint8_t posof[256];
    __shared__ uint32_t WP[8];
    __shared__ __align__(16) uint8_t seg[kTile];  // the segment's bytes, loaded at once
    const int b = blockIdx.y, g = blockIdx.x;
    const int m = st[b].m;
    const int s0 = g * kTile;
    if (s0 >= m) return;
    const int s1 = min(m, s0 + kTile);
    const int lane = threadIdx.x;
    {
        const uint8_t *Lb = L_all + (size_t)b * kBlockCap + s0;  // 16-byte aligned (block slots and tiles are)
        const int nb = s1 - s0;
        for (int q = lane; q < (nb >> 4); q += 32)
            reinterpret_cast<uint4 *>(seg)[q] = __ldg(reinterpret_cast<const uint4 *>(Lb) + q);
        for (int q = (nb & ~15) + lane; q < nb; q += 32) seg[q] = Lb[q];
    }
    if (lane < 8) iush[lane] = st[b].in_use[lane];
    __syncwarp();
    build_seq_table(iush, seq);
    int n_in_use = 0;
    for (int i = 0; i < 8; i++) n_in_use += __popc(iush[i]);
    const uint8_t *start = lists_all + ((size_t)b * kTilesPerBlock + g) * 256;
    for (int q = lane; q < 256; q += 32) lst[q] = start[q];
    __syncwarp();
    for (int q = lane; q < n_in_use; q += 32) posof[lst[q]] = (uint8_t)q;
    __syncwarp();
    uint8_t *out = idx_all + (size_t)b * kBlockCap;
    const uint32_t lt = lanemask_lt(), gt = lanemask_gt();
    for (int w0 = s0; w0 < s1; w0 += 32) {
        const int i = w0 + lane;
        const bool valid = i < s1;
        const uint32_t s = valid ? (uint32_t)seq[seg[i - s0]] : 256u + lane;
        const uint32_t grp = __match_any_sync(LFC_FULL, s);
        const uint32_t lower = grp & lt;
        const bool fo = valid && lower == 0;
        const uint32_t FO = __ballot_sync(LFC_FULL, fo);
        const uint32_t LAST = __ballot_sync(LFC_FULL, valid && (grp & gt) == 0);
        const uint32_t P = fo ? (uint32_t)posof[s] : 0u;
        const uint32_t maxP = __reduce_max_sync(LFC_FULL, P);
        const int pbits = 32 - __clz(maxP | 1u);  // bits of the deepest list position
        uint32_t gtm = 0, eqm = LFC_FULL;  // lanes with P_i > P
        for (int bb = pbits - 1; bb >= 0; bb--) {
            const uint32_t Bb = __ballot_sync(LFC_FULL, (P >> bb) & 1u);
            if ((P >> bb) & 1u) {
                eqm &= Bb;
            } else {
                gtm |= eqm & Bb;
                eqm &= ~Bb;
            }
        }
        const int j = lower ? 31 - __clz(lower) : -1;
        const uint32_t pp = lower ? (uint32_t)(j + 1) : 0u;  // prev + 1, in 0..31 (j <= 30)
        const uint32_t T = (uint32_t)(j + 1);
        uint32_t gt2 = 0, eq2 = LFC_FULL;  // lanes with prev_i + 1 > j + 1
#pragma unroll
        for (int bb = 4; bb >= 0; bb--) {
            const uint32_t Bb = __ballot_sync(LFC_FULL, (pp >> bb) & 1u);
            if ((T >> bb) & 1u) {
                eq2 &= Bb;
            } else {
                gt2 |= eq2 & Bb;
                eq2 &= ~Bb;
            }
        }
        uint32_t idx;
        if (lower == 0) idx = P + __popc(gtm & FO & lt);
        else idx = __popc(lt & ~((2u << j) - 1u) & ~gt2);
        if (valid) out[i] = (uint8_t)idx;
        // list update
        const uint32_t D = __popc(FO);
        if (lane < 8) WP[lane] = 0;
        __syncwarp();
        if (fo) atomicOr(&WP[P >> 5], 1u << (P & 31));
        __syncwarp();
        uint32_t mv[8];  // (new position << 8 | symbol) of the moved old entries, 0xFFFFFFFF if none
        uint32_t before = 0;  // window positions in earlier words
#pragma unroll
        for (int r = 0; r < 8; r++) {
            mv[r] = 0xFFFFFFFFu;
            const uint32_t q = (uint32_t)lane + 32u * r;
            if (32u * r > maxP) continue;
            const uint32_t wd = WP[r];
            if (q <= maxP && ((wd >> lane) & 1u) == 0) {
                const uint32_t rank = before + __popc(wd & lt);
                mv[r] = ((D + q - rank) << 8) | lst[q];
            }
            before += __popc(wd);
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < 8; r++) {
            if (mv[r] == 0xFFFFFFFFu) continue;
            const uint32_t np = mv[r] >> 8, x = mv[r] & 0xFFu;
            lst[np] = (uint8_t)x;
            posof[x] = (uint8_t)np;
        }
        if ((LAST >> lane) & 1u) {
            const uint32_t np = __popc(LAST & gt);
            lst[np] = (uint8_t)s;
            posof[s] = (uint8_t)np;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ RLE2
// Zero runs of length r -> bijective base-2 digits RUNA(0)/RUNB(1): digit k
// is bit k of r + 1, floor(log2(r + 1)) digits, emitted at the run's last
// position. Index j > 0 -> j + 1. As for RLE1, a scan over 4096-position
// tiles in three kernels: per tile the first / last nonzero index and the
// symbols of the positions after the first nonzero (1); per block the last
// nonzero before each tile, the symbols of each tile's leading zero run and
// the tiles' symbol offsets (2); per tile the symbols and their frequencies (3).
constexpr int kRle2Tile = 4096;
constexpr int kRle2Threads = 256;

__device__ __forceinline__ int run_digits(int r) { return 31 - __clz(r + 1); }

// Nonzero mask of a thread's 16 positions [a, a + 16) of the tile, a run-end
// mask (zero followed by a nonzero or by the end of the block) and the
// thread's first / last nonzero position (absolute; INT_MAX / -1 if none).
__device__ __forceinline__ void rle2_masks(const uint8_t *idx, int a, int te, int m, uint32_t &nz, uint32_t &end,
                                           int &first, int &last, uint8_t (&v)[16]) {
    *reinterpret_cast<uint4 *>(v) = *reinterpret_cast<const uint4 *>(idx + a);
    const uint32_t nxt = a + 16 < m ? idx[a + 16] : 0u;
    nz = 0; end = 0; first = INT_MAX; last = -1;
#pragma unroll
    for (int q = 0; q < 16; q++) {
        if (a + q >= te) break;
        if (v[q]) {
            nz |= 1u << q;
            first = min(first, a + q);
            last = a + q;
        } else {
            const bool next_nz = q < 15 ? (a + q + 1 < m && v[q + 1] != 0) : (a + 16 < m && nxt != 0);
            if (a + q == m - 1 || next_nz) end |= 1u << q;
        }
    }
}

__global__ void __launch_bounds__(kRle2Threads) rle2_tile_kernel(const BlockState *__restrict__ st,
                                                                 const uint8_t *__restrict__ idx_all,
                                                                 int32_t *__restrict__ aux_all) {
    __shared__ int sh[33];
    __shared__ int sfirst, slast;
    const int b = blockIdx.y, tile = blockIdx.x;
    const int m = st[b].m;
    const int ts = tile * kRle2Tile;
    if (ts >= m) return;
    const int te = min(m, ts + kRle2Tile);
    if (threadIdx.x == 0) { sfirst = INT_MAX; slast = -1; }
    const uint8_t *idx = idx_all + (size_t)b * kBlockCap;
    const int a = ts + 16 * (int)threadIdx.x;
    uint32_t nz = 0, end = 0;
    int first = INT_MAX, last = -1;
    uint8_t v[16];
    if (a < te) rle2_masks(idx, a, te, m, nz, end, first, last, v);
    int lz = block_excl_max(last, sh);   // last nonzero of the tile before this thread, or -1
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < 16; q++) {
        if ((nz >> q) & 1u) { cnt++; lz = a + q; }
        else if (((end >> q) & 1u) && lz >= ts) cnt += run_digits(a + q - lz);
    }
    int total;
    block_excl_sum<int>(cnt, sh, &total);
    if (first != INT_MAX) atomicMin(&sfirst, first);
    if (last >= 0) atomicMax(&slast, last);
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t *aux = aux_all + ((size_t)b * kTilesPerBlock + tile) * 4;
        aux[0] = sfirst != INT_MAX ? sfirst : te;
        aux[1] = slast;
        aux[2] = total;
    }
}

// One warp per block: aux[tile][1] = last nonzero before the tile (-1 if
// none), aux[tile][2] = the tile's symbol offset; symbol count, EOB and the
// frequency table's start.
__global__ void __launch_bounds__(32) rle2_scan_kernel(BlockState *__restrict__ st, int32_t *__restrict__ aux_all,
                                                       uint16_t *__restrict__ sym_all, uint32_t *__restrict__ freq_all) {
    const int b = blockIdx.x;
    const int m = st[b].m;
    const int ntile = (m + kRle2Tile - 1) / kRle2Tile;
    int32_t *aux = aux_all + (size_t)b * kTilesPerBlock * 4;
    const int lane = (int)lane_id();
    int carryR = -1, carryO = 0;
    for (int base = 0; base < ntile; base += 32) {
        const int t = base + lane;
        const bool valid = t < ntile;
        const int ts = t * kRle2Tile, te = min(m, ts + kRle2Tile);
        const int fs = valid ? aux[t * 4 + 0] : 0;
        const int ls = valid ? aux[t * 4 + 1] : -1;
        const int lo = valid ? aux[t * 4 + 2] : 0;
        const int imax = warp_incl_max(ls);
        int ex = __shfl_up_sync(LFC_FULL, imax, 1);
        if (lane == 0) ex = -1;
        const int R = max(carryR, ex);
        int pre = 0;  // the zero run the tile starts with, if it ends in the tile
        if (valid && fs > ts) {
            if (fs < te) {
                pre = run_digits(fs - 1 - R);
            } else if (te == m || (t + 1 < ntile && aux[(t + 1) * 4 + 0] == te)) {
                // no nonzero in the tile: the run ends at its last position when the
                // block ends there or the next tile starts with a nonzero
                pre = run_digits(te - 1 - R);
            }
        }
        const int out = valid ? pre + lo : 0;
        const int incl = warp_incl_sum(out);
        if (valid) {
            aux[t * 4 + 1] = R;
            aux[t * 4 + 2] = carryO + incl - out;
        }
        carryR = max(carryR, __shfl_sync(LFC_FULL, imax, 31));
        carryO += __shfl_sync(LFC_FULL, incl, 31);
    }
    int n_in_use = 0;
    for (int i = 0; i < 8; i++) n_in_use += __popc(st[b].in_use[i]);
    uint32_t *freq = freq_all + (size_t)b * kMaxAlpha;
    for (int i = lane; i < kMaxAlpha; i += 32) freq[i] = i == n_in_use + 1 ? 1u : 0u;
    if (lane == 0) {
        sym_all[(size_t)b * kSymStride + carryO] = (uint16_t)(n_in_use + 1);
        st[b].n_mtf = carryO + 1;
        st[b].n_in_use = n_in_use;
    }
}

__global__ void __launch_bounds__(kRle2Threads) rle2_write_kernel(const BlockState *__restrict__ st,
                                                                  const uint8_t *__restrict__ idx_all,
                                                                  const int32_t *__restrict__ aux_all,
                                                                  uint16_t *__restrict__ sym_all, uint32_t *__restrict__ freq_all) {
    __shared__ int sh[33];
    __shared__ uint32_t fq[kMaxAlpha];
    // the tile's symbols: a zero run of r codes to at most r digits, and only
    // the first run ending in the tile can hold zeros of earlier tiles (at
    // most 20 digits: a block is below 2^20 positions)
    __shared__ uint16_t ssym[kRle2Tile + 32];
    const int b = blockIdx.y, tile = blockIdx.x;
    const int m = st[b].m;
    const int ts = tile * kRle2Tile;
    if (ts >= m) return;
    const int te = min(m, ts + kRle2Tile);
    for (int i = threadIdx.x; i < kMaxAlpha; i += kRle2Threads) fq[i] = 0;
    const uint8_t *idx = idx_all + (size_t)b * kBlockCap;
    const int32_t *aux = aux_all + ((size_t)b * kTilesPerBlock + tile) * 4;
    const int R = aux[1], off = aux[2];
    const int a = ts + 16 * (int)threadIdx.x;
    uint32_t nz = 0, end = 0;
    int first = INT_MAX, last = -1;
    uint8_t v[16];
    if (a < te) rle2_masks(idx, a, te, m, nz, end, first, last, v);
    const int lz0 = max(block_excl_max(last, sh), R);
    int lz = lz0, cnt = 0;
#pragma unroll
    for (int q = 0; q < 16; q++) {
        if ((nz >> q) & 1u) { cnt++; lz = a + q; }
        else if ((end >> q) & 1u) cnt += run_digits(a + q - lz);
    }
    // symbols staged in shared memory at their tile-local offsets, then
    // written by consecutive threads on consecutive positions
    int total = 0;
    int o = block_excl_sum<int>(cnt, sh, &total);
    uint16_t *sym = sym_all + (size_t)b * kSymStride;
    lz = lz0;
#pragma unroll
    for (int q = 0; q < 16; q++) {
        if ((nz >> q) & 1u) {
            const uint32_t s = (uint32_t)v[q] + 1u;
            ssym[o++] = (uint16_t)s;
            atomicAdd(&fq[s], 1u);
            lz = a + q;
        } else if ((end >> q) & 1u) {
            const uint32_t r1 = (uint32_t)(a + q - lz);  // run length r, digits of r + 1
            const int nd = run_digits((int)r1);
            for (int k = 0; k < nd; k++) {
                const uint32_t d = ((r1 + 1u) >> k) & 1u;
                ssym[o++] = (uint16_t)d;
                atomicAdd(&fq[d], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < total; i += kRle2Threads) sym[off + i] = ssym[i];
    uint32_t *freq = freq_all + (size_t)b * kMaxAlpha;
    for (int i = threadIdx.x; i < kMaxAlpha; i += kRle2Threads)
        if (fq[i]) atomicAdd(&freq[i], fq[i]);
}

// --------------------------------------------------------------- Huffman
// Code lengths of one table by one warp: weights max(freq, 1); the two nodes
// with the smallest (weight, key) are joined (leaf key = symbol, k-th joined
// node key = alpha + k; the two-queue method reproduces that order because
// leaves are pre-sorted by (weight, symbol) and joined nodes appear in
// non-decreasing weight); over-long codes halve the weights (1 + w/2).
struct HuffScratch {
    uint32_t w[kMaxAlpha];
    uint32_t lw[kMaxAlpha];          // leaf weights in (weight, symbol) order
    uint32_t nw[kMaxAlpha];          // joined-node weights
    uint16_t order[kMaxAlpha];       // leaves sorted by (w, symbol)
    uint16_t par[2 * kMaxAlpha];     // parent of a node (leaves, then joined nodes)
    uint16_t dist[2 * kMaxAlpha];    // pointer-jumping distance to par
};

// Keys (w << 9 | symbol) are distinct, so a key's rank is the count of
// smaller keys; w < 2^21 (counts of one block), so the key fits 30 bits.
// Node depths by pointer jumping: after r rounds par[n] is n's 2^r-th
// ancestor (capped at the root) and dist[n] the distance to it; 9 rounds
// cover depths up to 511 >= alpha - 1.
__device__ void huff_lengths_warp(const uint32_t *freq, int alpha, int max_len, uint8_t *len_out, HuffScratch &S) {
    constexpr int kQ = (kMaxAlpha + 31) / 32;       // leaves per lane
    constexpr int kN = (2 * kMaxAlpha + 31) / 32;   // nodes per lane
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < alpha; i += 32) S.w[i] = freq[i] ? freq[i] : 1u;
    __syncwarp();
    const int nodes = 2 * alpha - 1, root = 2 * alpha - 2;
    int longest = 0;
    for (;;) {
        uint32_t myk[kQ], rk[kQ];
#pragma unroll
        for (int q = 0; q < kQ; q++) {
            const int i = lane + 32 * q;
            myk[q] = i < alpha ? ((S.w[i] << 9) | (uint32_t)i) : 0xFFFFFFFFu;
            rk[q] = 0;
        }
        for (int j = 0; j < alpha; j++) {
            const uint32_t kj = (S.w[j] << 9) | (uint32_t)j;
#pragma unroll
            for (int q = 0; q < kQ; q++) rk[q] += kj < myk[q];
        }
#pragma unroll
        for (int q = 0; q < kQ; q++) {
            const int i = lane + 32 * q;
            if (i < alpha) {
                S.order[rk[q]] = (uint16_t)i;
                S.lw[rk[q]] = S.w[i];
            }
        }
        __syncwarp();
        if (lane == 0) {
            // two-queue merge: the two smallest (weight, key) nodes, a leaf
            // before a joined node of equal weight (its key is smaller)
            int la = 0, lb = 0, nb = 0;
            uint32_t ha = S.lw[0], hb = 0;
            for (int k = 0; k < alpha - 1; k++) {
                int pick[2];
                uint32_t pw[2];
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const bool takeA = lb >= nb || (la < alpha && ha <= hb);
                    if (takeA) {
                        pick[q] = S.order[la];
                        pw[q] = ha;
                        la++;
                        ha = la < alpha ? S.lw[la] : 0u;
                    } else {
                        pick[q] = alpha + lb;
                        pw[q] = hb;
                        lb++;
                        hb = lb < nb ? S.nw[lb] : 0u;
                    }
                }
                const uint32_t sw = pw[0] + pw[1];
                S.par[pick[0]] = (uint16_t)(alpha + k);
                S.par[pick[1]] = (uint16_t)(alpha + k);
                S.nw[nb] = sw;
                if (lb == nb) hb = sw;  // the joined queue was empty
                nb++;
            }
            S.par[root] = (uint16_t)root;
        }
        __syncwarp();
        uint16_t pn[kN], dn[kN];
#pragma unroll
        for (int q = 0; q < kN; q++) {
            const int n = lane + 32 * q;
            if (n < nodes) S.dist[n] = n == root ? 0 : 1;
        }
        __syncwarp();
        for (int round = 0; round < 9; round++) {
#pragma unroll
            for (int q = 0; q < kN; q++) {
                const int n = lane + 32 * q;
                if (n < nodes) {
                    const int pp = S.par[n];
                    dn[q] = (uint16_t)(S.dist[n] + S.dist[pp]);
                    pn[q] = S.par[pp];
                }
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < kN; q++) {
                const int n = lane + 32 * q;
                if (n < nodes) {
                    S.dist[n] = dn[q];
                    S.par[n] = pn[q];
                }
            }
            __syncwarp();
        }
        int mx = 0;
        for (int i = lane; i < alpha; i += 32) mx = max(mx, (int)S.dist[i]);
        longest = __reduce_max_sync(LFC_FULL, (unsigned)mx);
        if (longest <= max_len) break;
        for (int i = lane; i < alpha; i += 32) S.w[i] = 1u + S.w[i] / 2u;
        __syncwarp();
    }
    for (int i = lane; i < alpha; i += 32) len_out[i] = (uint8_t)S.dist[i];
    __syncwarp();
}

constexpr int kPackGroups = 128;                                           // selector groups per tile = threads
constexpr int kPackTiles = (kMaxSelectors + kPackGroups - 1) / kPackGroups;  // 141
constexpr int kTileSyms = kPackGroups * 50;                                   // symbols of a tile

// Stage the symbols of a tile of selector groups in shared memory with
// coalesced 16-byte loads (tile starts are 16-byte aligned); returns their count.
__device__ __forceinline__ int stage_tile_syms(const uint16_t *sym, int tile, int n_mtf, uint16_t *ssym) {
    const int a = tile * kTileSyms;
    const int cnt = min(kTileSyms, n_mtf - a);
    const int n8 = cnt >> 3;
    const uint4 *src = reinterpret_cast<const uint4 *>(sym + a);
    uint4 *dst = reinterpret_cast<uint4 *>(ssym);
    for (int i = threadIdx.x; i < n8; i += blockDim.x) dst[i] = src[i];
    for (int i = (n8 << 3) + threadIdx.x; i < cnt; i += blockDim.x) ssym[i] = sym[a + i];
    return cnt;
}

// Table choice per block, in launches: the table count and the initial
// partition by cumulative frequency (init); four refinement passes, each
// "every 50-symbol group picks the cheapest table, ties to the lower" over
// many CTAs (select) followed by "every table is rebuilt from its groups'
// counts with a 17-bit limit" (build); canonical codes (codes).
constexpr int kHuffBuildThreads = 32 * kMaxGroups;

__global__ void __launch_bounds__(256) huff_init_kernel(BlockState *__restrict__ st, const uint32_t *__restrict__ freq_all,
                                                        uint8_t *__restrict__ lens_all, uint32_t *__restrict__ rfreq_all) {
    const int b = blockIdx.x;
    const int n_mtf = st[b].n_mtf;
    const int alpha = st[b].n_in_use + 2;
    const int ng = n_mtf < 200 ? 2 : n_mtf < 600 ? 3 : n_mtf < 1200 ? 4 : n_mtf < 2400 ? 5 : 6;
    for (int i = threadIdx.x; i < kMaxGroups * kMaxAlpha; i += blockDim.x) rfreq_all[(size_t)b * kMaxGroups * kMaxAlpha + i] = 0;
    if (threadIdx.x == 0) {
        const uint32_t *freq = freq_all + (size_t)b * kMaxAlpha;
        uint8_t *len = lens_all + (size_t)b * kMaxGroups * kMaxAlpha;
        int64_t cum = 0;
        for (int v = 0; v < alpha; v++) {
            int64_t gsel = cum * ng / n_mtf;
            if (gsel > ng - 1) gsel = ng - 1;
            for (int t = 0; t < ng; t++) len[t * kMaxAlpha + v] = (uint8_t)(t == gsel ? 0 : 15);
            cum += freq[v];
        }
        st[b].n_groups = ng;
        st[b].n_sel = (n_mtf + 49) / 50;
    }
}

// Thread per 50-symbol group: cost under every table (10-bit fields of one
// 64-bit word per symbol; <= 50 x 17 bits), the cheapest table, and the
// group's symbols added to that table's counts (RUNA / RUNB, the most common
// symbols, in registers; the rest through shared memory, flushed per CTA).
__global__ void __launch_bounds__(kPackGroups) huff_select_kernel(const BlockState *__restrict__ st,
                                                                  const uint16_t *__restrict__ sym_all,
                                                                  const uint8_t *__restrict__ lens_all,
                                                                  uint8_t *__restrict__ sel_all, uint32_t *__restrict__ rfreq_all) {
    __shared__ uint64_t packed[kMaxAlpha];
    __shared__ uint32_t rf[kMaxGroups][kMaxAlpha];
    __shared__ __align__(16) uint16_t ssym[kTileSyms];
    const int b = blockIdx.y, tile = blockIdx.x;
    const BlockState S = st[b];
    const int ng = S.n_groups, nsel = S.n_sel, n_mtf = S.n_mtf, alpha = S.n_in_use + 2;
    if (tile * kPackGroups >= nsel) return;
    stage_tile_syms(sym_all + (size_t)b * kSymStride, tile, n_mtf, ssym);
    const uint8_t *len = lens_all + (size_t)b * kMaxGroups * kMaxAlpha;
    for (int v = threadIdx.x; v < alpha; v += blockDim.x) {
        uint64_t pk = 0;
        for (int t = 0; t < ng; t++) pk |= (uint64_t)len[t * kMaxAlpha + v] << (10 * t);
        packed[v] = pk;
    }
    for (int i = threadIdx.x; i < kMaxGroups * kMaxAlpha; i += blockDim.x) (&rf[0][0])[i] = 0;
    __syncthreads();
    const int gi = tile * kPackGroups + (int)threadIdx.x;
    int bt = -1;
    uint32_t c0 = 0, c1 = 0;
    if (gi < nsel) {
        const uint16_t *sym = ssym - tile * kTileSyms;  // indexed by block position
        const int a = gi * 50, e = min(n_mtf, a + 50);
        uint64_t acc = 0;
        for (int i = a; i < e; i++) acc += packed[sym[i]];
        bt = 0;
        uint32_t bc = (uint32_t)(acc & 1023u);
        for (int t = 1; t < ng; t++) {
            const uint32_t c = (uint32_t)((acc >> (10 * t)) & 1023u);
            if (c < bc) { bc = c; bt = t; }
        }
        sel_all[(size_t)b * kMaxSelectors + gi] = (uint8_t)bt;
        for (int i = a; i < e; i++) {
            const uint32_t v = sym[i];
            if (v == 0) c0++;
            else if (v == 1) c1++;
            else atomicAdd(&rf[bt][v], 1u);
        }
        if (c0) atomicAdd(&rf[bt][0], c0);
        if (c1) atomicAdd(&rf[bt][1], c1);
    }
    __syncthreads();
    uint32_t *rfreq = rfreq_all + (size_t)b * kMaxGroups * kMaxAlpha;
    for (int i = threadIdx.x; i < ng * kMaxAlpha; i += blockDim.x) {
        const uint32_t c = (&rf[0][0])[i];
        if (c) atomicAdd(&rfreq[i], c);
    }
}

// Warp per table: code lengths from the pass's counts, which are then
// cleared for the next pass.
__global__ void __launch_bounds__(kHuffBuildThreads) huff_build_kernel(const BlockState *__restrict__ st,
                                                                       uint32_t *__restrict__ rfreq_all,
                                                                       uint8_t *__restrict__ lens_all) {
    __shared__ uint32_t cnt[kMaxGroups][kMaxAlpha];
    __shared__ uint8_t lo[kMaxGroups][kMaxAlpha];
    __shared__ HuffScratch scratch[kMaxGroups];
    const int b = blockIdx.x;
    const int ng = st[b].n_groups, alpha = st[b].n_in_use + 2;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w >= ng) return;
    uint32_t *rfreq = rfreq_all + ((size_t)b * kMaxGroups + w) * kMaxAlpha;
    for (int v = lane; v < alpha; v += 32) {
        cnt[w][v] = rfreq[v];
        rfreq[v] = 0;
    }
    __syncwarp();
    huff_lengths_warp(cnt[w], alpha, 17, lo[w], scratch[w]);
    uint8_t *len = lens_all + ((size_t)b * kMaxGroups + w) * kMaxAlpha;
    for (int v = lane; v < alpha; v += 32) len[v] = lo[w][v];
}

// Canonical codes: by length, then symbol (lane 0 of the table's warp).
__global__ void __launch_bounds__(kHuffBuildThreads) huff_codes_kernel(const BlockState *__restrict__ st,
                                                                       const uint8_t *__restrict__ lens_all,
                                                                       uint32_t *__restrict__ codes_all) {
    const int b = blockIdx.x;
    const int ng = st[b].n_groups, alpha = st[b].n_in_use + 2;
    const int w = threadIdx.x >> 5;
    if (w >= ng || (threadIdx.x & 31) != 0) return;
    const uint8_t *len = lens_all + ((size_t)b * kMaxGroups + w) * kMaxAlpha;
    uint32_t next[22];
    uint32_t cnt[22];
    for (int l = 0; l < 22; l++) cnt[l] = 0;
    for (int v = 0; v < alpha; v++) cnt[len[v]]++;
    uint32_t c = 0;
    for (int l = 1; l <= 20; l++) { next[l] = c; c = (c + cnt[l]) << 1; }
    uint32_t *codes = codes_all + ((size_t)b * kMaxGroups + w) * kMaxAlpha;
    for (int v = 0; v < alpha; v++) codes[v] = next[len[v]]++;
}

// ------------------------------------------------------------ bit packing
// Bits are numbered from the start of the stream; bit P lands in word P/32 at
// bit 31 - P%32 (MSB first). Words are stored byte-swapped (so the bytes
// come out in stream order); swapping commutes with OR, so partial words
// from different writers are swapped first and OR-ed into zeroed memory.
__device__ __forceinline__ uint32_t bswap32(uint32_t w) { return __byte_perm(w, 0u, 0x0123); }

__device__ __forceinline__ void put_bits(uint32_t *words, uint64_t pos, uint32_t value, int nbits) {
    if (nbits == 0) return;
    const int sh = (int)(pos & 31);
    const uint64_t v = (uint64_t)value << (64 - nbits - sh);
    const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
    if (hi) atomicOr(&words[pos >> 5], bswap32(hi));
    if (lo) atomicOr(&words[(pos >> 5) + 1], bswap32(lo));
}

// MTF index of a selector of table s (tables listed 0..ng-1 initially),
// given last[t] = position of the latest earlier selector of table t (-1 if
// none): the number of tables used since s was last used, or, before its
// first use, the tables used so far plus the unused tables below s.
__device__ __forceinline__ int selector_mtf(int s, const int (&last)[kMaxGroups], int ng) {
    int ls = -1;
#pragma unroll
    for (int t = 0; t < kMaxGroups; t++)
        if (t == s) ls = last[t];
    int j = 0;
#pragma unroll
    for (int t = 0; t < kMaxGroups; t++) {
        if (t >= ng || t == s) continue;
        j += ls >= 0 ? (last[t] > ls) : (last[t] >= 0 || t < s);
    }
    return j;
}

__device__ __forceinline__ void set_last(int (&last)[kMaxGroups], int s, int i) {
#pragma unroll
    for (int t = 0; t < kMaxGroups; t++)
        if (t == s) last[t] = i;
}

// Data packing is a scan over tiles of 128 selector groups (50 symbols each):
// group bit lengths and tile sums (1); per block the stream layout, the tile
// offsets, the header, selector, code-length and trailer sections (2); each
// group's codes from its bit offset, whole words stored, the two boundary
// words OR-ed (3).
static_assert(kPackTiles <= kTilesPerBlock, "pack tile records live in the per-block tile scratch");
constexpr int kLayoutThreads = 1024;

__device__ __forceinline__ void load_tables(const uint8_t *lens_all, const uint32_t *codes_all, int b, int ng,
                                            uint8_t (*len)[kMaxAlpha], uint32_t (*code)[kMaxAlpha]) {
    for (int i = threadIdx.x; i < ng * kMaxAlpha; i += blockDim.x) {
        const int t = i / kMaxAlpha, v = i - t * kMaxAlpha;
        len[t][v] = lens_all[((size_t)b * kMaxGroups + t) * kMaxAlpha + v];
        if (code) code[t][v] = codes_all[((size_t)b * kMaxGroups + t) * kMaxAlpha + v];
    }
}

__global__ void __launch_bounds__(kPackGroups) pack_bits_kernel(const BlockState *__restrict__ st,
                                                                const uint16_t *__restrict__ sym_all,
                                                                const uint8_t *__restrict__ sel_all,
                                                                const uint8_t *__restrict__ lens_all,
                                                                uint16_t *__restrict__ gbits_all,
                                                                int32_t *__restrict__ aux_all) {
    __shared__ uint8_t len[kMaxGroups][kMaxAlpha];
    __shared__ int sh[33];
    __shared__ __align__(16) uint16_t ssym[kTileSyms];
    const int b = blockIdx.y, tile = blockIdx.x;
    const BlockState S = st[b];
    if (tile * kPackGroups >= S.n_sel) return;
    load_tables(lens_all, nullptr, b, S.n_groups, len, nullptr);
    stage_tile_syms(sym_all + (size_t)b * kSymStride, tile, S.n_mtf, ssym);
    __syncthreads();
    const int gi = tile * kPackGroups + (int)threadIdx.x;
    int bits = 0;
    if (gi < S.n_sel) {
        const uint16_t *sym = ssym - tile * kTileSyms;
        const uint8_t *lt = len[sel_all[(size_t)b * kMaxSelectors + gi]];
        const int a = gi * 50, e = min(S.n_mtf, a + 50);
        for (int i = a; i < e; i++) bits += lt[sym[i]];
        gbits_all[(size_t)b * (kBlockCap / 2) + gi] = (uint16_t)bits;
    }
    int total;
    block_excl_sum<int>(bits, sh, &total);
    if (threadIdx.x == 0) aux_all[((size_t)b * kTilesPerBlock + tile) * 4] = total;
}

__global__ void __launch_bounds__(kLayoutThreads) pack_layout_kernel(BlockState *__restrict__ st,
                                                                     const uint8_t *__restrict__ sel_all,
                                                                     const uint8_t *__restrict__ lens_all,
                                                                     int32_t *__restrict__ aux_all,
                                                                     uint32_t *__restrict__ packed_all, int64_t stream_words) {
    __shared__ uint8_t len[kMaxGroups][kMaxAlpha];
    __shared__ uint64_t sh64[33];
    __shared__ int shi[33];
    __shared__ uint32_t tbl_bits[kMaxGroups];
    __shared__ uint64_t base_bits[4];
    const int b = blockIdx.x;
    const BlockState S = st[b];
    const int ng = S.n_groups, nsel = S.n_sel, alpha = S.n_in_use + 2;
    const uint8_t *sel = sel_all + (size_t)b * kMaxSelectors;
    uint32_t *words = packed_all + (size_t)b * stream_words;
    int32_t *aux = aux_all + (size_t)b * kTilesPerBlock * 4;
    load_tables(lens_all, nullptr, b, ng, len, nullptr);
    uint32_t used16 = 0;
    for (int i = 0; i < 16; i++) {
        const uint32_t half = (S.in_use[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu;
        if (half) used16 |= 1u << (15 - i);
    }
    __syncthreads();
    // data tiles: exclusive offsets (one tile per thread, <= 141 tiles)
    const int ntiles = (nsel + kPackGroups - 1) / kPackGroups;
    const uint64_t tb = (int)threadIdx.x < ntiles ? (uint64_t)(uint32_t)aux[threadIdx.x * 4] : 0ull;
    uint64_t data_total;
    const uint64_t toff = block_excl_sum<uint64_t>(tb, sh64, &data_total);
    if ((int)threadIdx.x < ntiles) aux[threadIdx.x * 4 + 1] = (int32_t)toff;
    // selector MTF: each thread's span starts from the last use of every table
    // before it (exclusive max-scans), then replays its span
    const int T = blockDim.x;
    const int sper = (nsel + T - 1) / T;
    const int sa = min(nsel, (int)threadIdx.x * sper), se = min(nsel, sa + sper);
    int last0[kMaxGroups];
#pragma unroll
    for (int t = 0; t < kMaxGroups; t++) last0[t] = -1;
    for (int i = sa; i < se; i++) set_last(last0, sel[i], i);
#pragma unroll
    for (int t = 0; t < kMaxGroups; t++) last0[t] = block_excl_max(last0[t], shi);
    int last[kMaxGroups];
#pragma unroll
    for (int t = 0; t < kMaxGroups; t++) last[t] = last0[t];
    uint64_t sbits = 0;
    for (int i = sa; i < se; i++) {
        const int sv = sel[i];
        sbits += (uint64_t)selector_mtf(sv, last, ng) + 1;
        set_last(last, sv, i);
    }
    uint64_t sel_total;
    const uint64_t sel_off = block_excl_sum<uint64_t>(sbits, sh64, &sel_total);
    // code-length section bits per table (warp t)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < ng) {
        uint32_t bits = 0;
        for (int v = lane; v < alpha; v += 32) {
            const int d = v == 0 ? 0 : (int)len[w][v] - (int)len[w][v - 1];
            bits += 2u * (uint32_t)abs(d) + 1u;
        }
        bits = warp_sum(bits);
        if (lane == 0) tbl_bits[w] = bits + 5u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t p = 32 + 48 + 32 + 1 + 24 + 16 + 16ull * __popc(used16) + 3 + 15;
        base_bits[0] = p;                       // selectors start
        p += sel_total;
        for (int t = 0; t < ng; t++) p += tbl_bits[t];
        base_bits[1] = p;                       // data start
        p += data_total;
        base_bits[2] = p;                       // trailer start
        p += 48 + 32;
        p = (p + 7) & ~7ull;
        base_bits[3] = p;                       // total bits
    }
    __syncthreads();
    const uint64_t total_bits = base_bits[3];
    const int64_t nwords = (int64_t)((total_bits + 31) >> 5);
    for (int64_t i = threadIdx.x; i < nwords + 1 && i < stream_words; i += blockDim.x) words[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t p = 0;
        put_bits(words, p, 0x425A6839u, 32); p += 32;  // "BZh9"
        put_bits(words, p, 0x314159u, 24); p += 24;
        put_bits(words, p, 0x265359u, 24); p += 24;
        put_bits(words, p, S.crc, 32); p += 32;
        put_bits(words, p, 0, 1); p += 1;
        put_bits(words, p, (uint32_t)S.orig_ptr, 24); p += 24;
        put_bits(words, p, used16, 16); p += 16;
        for (int i = 0; i < 16; i++) {
            if (!(used16 & (1u << (15 - i)))) continue;
            const uint32_t half = (S.in_use[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu;
            put_bits(words, p, __brev(half) >> 16, 16);  // byte 16i+j -> bit 15-j
            p += 16;
        }
        put_bits(words, p, (uint32_t)ng, 3); p += 3;
        put_bits(words, p, (uint32_t)nsel, 15); p += 15;
        uint64_t q = base_bits[2];
        put_bits(words, q, 0x177245u, 24); q += 24;
        put_bits(words, q, 0x385090u, 24); q += 24;
        put_bits(words, q, S.crc, 32);
        st[b].stream_bits = (uint32_t)total_bits;
        st[b].stream_bytes = (uint32_t)(total_bits >> 3);
        st[b].data_bit0 = (uint32_t)base_bits[1];
    }
    {   // selectors: j ones then a zero
        uint64_t p = base_bits[0] + sel_off;
        for (int t = 0; t < kMaxGroups; t++) last[t] = last0[t];
        for (int i = sa; i < se; i++) {
            const int sv = sel[i];
            const int j = selector_mtf(sv, last, ng);
            set_last(last, sv, i);
            put_bits(words, p, ((1u << j) - 1u) << 1, j + 1);
            p += (uint64_t)j + 1;
        }
    }
    if (w < ng) {  // code lengths: 5-bit start, then per symbol |d| x ("10" up or "11" down) and a '0'
        uint64_t p = base_bits[0] + sel_total;
        for (int t = 0; t < w; t++) p += tbl_bits[t];
        if (lane == 0) put_bits(words, p, (uint32_t)len[w][0], 5);
        p += 5;
        for (int v0 = 0; v0 < alpha; v0 += 32) {
            const int v = v0 + lane;
            const int d = v < alpha ? (v == 0 ? 0 : (int)len[w][v] - (int)len[w][v - 1]) : 0;
            const uint32_t nb = v < alpha ? 2u * (uint32_t)abs(d) + 1u : 0u;
            const uint32_t incl = warp_incl_sum(nb);
            uint64_t q = p + incl - nb;
            for (int k = 0; k < abs(d); k++, q += 2) put_bits(words, q, d > 0 ? 2u : 3u, 2);
            p += __shfl_sync(LFC_FULL, incl, 31);
        }
    }
}

__global__ void __launch_bounds__(kPackGroups) pack_data_kernel(const BlockState *__restrict__ st,
                                                                const uint16_t *__restrict__ sym_all,
                                                                const uint8_t *__restrict__ sel_all,
                                                                const uint8_t *__restrict__ lens_all,
                                                                const uint32_t *__restrict__ codes_all,
                                                                const uint16_t *__restrict__ gbits_all,
                                                                const int32_t *__restrict__ aux_all,
                                                                uint32_t *__restrict__ packed_all, int64_t stream_words) {
    __shared__ uint8_t len[kMaxGroups][kMaxAlpha];
    __shared__ uint32_t code[kMaxGroups][kMaxAlpha];
    __shared__ int sh[33];
    __shared__ __align__(16) uint16_t ssym[kTileSyms];
    const int b = blockIdx.y, tile = blockIdx.x;
    const BlockState S = st[b];
    if (tile * kPackGroups >= S.n_sel) return;
    load_tables(lens_all, codes_all, b, S.n_groups, len, code);
    stage_tile_syms(sym_all + (size_t)b * kSymStride, tile, S.n_mtf, ssym);
    const int gi = tile * kPackGroups + (int)threadIdx.x;
    const int bits = gi < S.n_sel ? (int)gbits_all[(size_t)b * (kBlockCap / 2) + gi] : 0;
    const int off = block_excl_sum<int>(bits, sh, nullptr);  // also orders the table loads
    if (gi >= S.n_sel || bits == 0) return;
    uint32_t *words = packed_all + (size_t)b * stream_words;
    const uint64_t p0 = (uint64_t)S.data_bit0 + (uint32_t)aux_all[((size_t)b * kTilesPerBlock + tile) * 4 + 1] + off;
    const int t = sel_all[(size_t)b * kMaxSelectors + gi];
    const uint16_t *sym = ssym - tile * kTileSyms;
    const int a = gi * 50, e = min(S.n_mtf, a + 50);
    uint64_t acc = 0;                 // pending bits, left-aligned
    uint64_t wpos = p0 & ~31ull;      // bit position of the word being built
    int nacc = (int)(p0 - wpos);      // leading bits owned by the previous group (zeros)
    for (int i = a; i < e; i++) {
        const uint32_t sv = sym[i];
        const int l = len[t][sv];
        acc |= (uint64_t)code[t][sv] << (64 - nacc - l);
        nacc += l;
        if (nacc >= 32) {
            const uint32_t word = bswap32((uint32_t)(acc >> 32));
            if (wpos < p0) atomicOr(&words[wpos >> 5], word);  // shared with the previous group
            else words[wpos >> 5] = word;
            acc <<= 32;
            nacc -= 32;
            wpos += 32;
        }
    }
    if (nacc > 0) atomicOr(&words[wpos >> 5], bswap32((uint32_t)(acc >> 32)));  // shared with the next
}

cudaError_t launch_mtf_rle2(lfc_plan P, int nblocks) {
    Workspace &ws = P->ws;
    cudaStream_t s = P->stream;
    dim3 grid(kTilesPerBlock, nblocks);
    mtf_compose_kernel<<<nblocks, 256, 0, s>>>(ws.bstate, ws.mtfrec, ws.mtfreclen, ws.mtflists);
    mtf_encode_kernel<<<grid, 32, 0, s>>>(ws.bstate, ws.bwt, ws.mtflists, ws.mtfidx);
    const dim3 g2(kTilesPerBlock, nblocks);  // RLE1 output <= 900000 = 220 tiles
    rle2_tile_kernel<<<g2, kRle2Threads, 0, s>>>(ws.bstate, ws.mtfidx, ws.tileaux);
    rle2_scan_kernel<<<nblocks, 32, 0, s>>>(ws.bstate, ws.tileaux, ws.sym, ws.freq);
    rle2_write_kernel<<<g2, kRle2Threads, 0, s>>>(ws.bstate, ws.mtfidx, ws.tileaux, ws.sym, ws.freq);
    count_launches(P, 5);
    return cudaGetLastError();
}

cudaError_t launch_huffman(lfc_plan P, int nblocks) {
    Workspace &ws = P->ws;
    cudaStream_t s = P->stream;
    huff_init_kernel<<<nblocks, 256, 0, s>>>(ws.bstate, ws.freq, ws.lens, ws.rfreq);
    const dim3 grid(kPackTiles, nblocks);
    for (int iter = 0; iter < 4; iter++) {
        huff_select_kernel<<<grid, kPackGroups, 0, s>>>(ws.bstate, ws.sym, ws.lens, ws.sel, ws.rfreq);
        huff_build_kernel<<<nblocks, kHuffBuildThreads, 0, s>>>(ws.bstate, ws.rfreq, ws.lens);
    }
    huff_codes_kernel<<<nblocks, kHuffBuildThreads, 0, s>>>(ws.bstate, ws.lens, ws.codes);
    count_launches(P, 10);
    return cudaGetLastError();
}

cudaError_t launch_pack(lfc_plan P, int nblocks) {
    Workspace &ws = P->ws;
    // group bit lengths live in the MTF index slots, free once RLE2 has run
    uint16_t *gbits = reinterpret_cast<uint16_t *>(ws.mtfidx);
    const dim3 grid(kPackTiles, nblocks);
    pack_bits_kernel<<<grid, kPackGroups, 0, P->stream>>>(ws.bstate, ws.sym, ws.sel, ws.lens, gbits, ws.tileaux);
    pack_layout_kernel<<<nblocks, kLayoutThreads, 0, P->stream>>>(ws.bstate, ws.sel, ws.lens, ws.tileaux, ws.packed,
                                                                  ws.stream_words);
    pack_data_kernel<<<grid, kPackGroups, 0, P->stream>>>(ws.bstate, ws.sym, ws.sel, ws.lens, ws.codes, gbits,
                                                          ws.tileaux, ws.packed, ws.stream_words);
    count_launches(P, 3);
    return cudaGetLastError();
}

}  // namespace lfc

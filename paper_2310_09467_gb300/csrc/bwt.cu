// bwt.cu -- RLE1 and the Burrows-Wheeler transform of every bzip2 block
// (Sec. 2.1.3 codes the chosen stream with bzip2; the block format is the
// public bzip2 format).
//
// BWT = sort of all cyclic rotations, ties between identical rotations by
// start index. Two phases over all blocks of a pass at once, one CTA per
// (4096-element tile, block), block-major so a block's data stays in L2
// while its tiles run. Every element carries its sort key: a radix pass
// reads (key, element) pairs coalesced, ranks each tile by digit in shared
// memory and writes each digit's run of the tile contiguously.
//  1. Keys = the first 8 bytes of each rotation (big-endian), built from
//     sequential reads; 8 stable LSD passes of 8-bit digits.
//  2. Prefix doubling on the groups still tied: rank[i] = head position of
//     i's group in the suffix array; each round keys the tied elements by
//     (rank[i] << 20 | rank[i + h]) (m < 2^20), sorts them with 5 stable LSD
//     passes, splits groups, and doubles h. Here an element is one 64-bit
//     word, the 40-bit key above the element (20 bits), and the passes sort
//     bits 20..59 only. Groups left when h >= m hold identical rotations,
//     already in start-index order (every pass is stable and the first starts
//     from the identity).
#include <climits>
#include <utility>

#ifndef LFC_PHASE1_BYTES
#define LFC_PHASE1_BYTES 8
#endif

#include "lfc_common.cuh"

namespace lfc {

constexpr int kSortThreads = 256;
constexpr int kPerThread = kTile / kSortThreads;  // 16

// ------------------------------------------------------------------ RLE1
// A run of L equal bytes is cut into 255-byte pieces; a piece of 4 or more
// bytes becomes its first 4 bytes and a count byte (length - 4), a shorter
// one stays literal. So the byte at offset k of its run adds w(k mod 255)
// output bytes, w = 1, 1, 1, 2, 0, 0, ... (the fourth byte carries the count
// byte), and a run of L bytes codes to G(L) = sum_{k<L} w(k mod 255) bytes.
// That makes RLE1 a scan over 4096-byte tiles of every block, in three
// kernels: per tile the first / last run start and the output of the
// positions whose run starts inside the tile (1); per block, in tile order,
// the run start carried into each tile and the tile's output offset (2); per
// tile, every position's output offset and its bytes, staged in shared
// memory and stored coalesced (3).
constexpr int kRleTile = 4096;
constexpr int kRleThreads = 256;                  // 16 bytes per thread
constexpr int kRleMaxTiles = (LFC_MAX_BLOCK_BYTES + kRleTile - 1) / kRleTile;
constexpr int kRleOutCap = kRleTile / 4 * 5 + 16; // at most 5 output bytes per 4 inputs, + edge
static_assert(kRleMaxTiles <= kTilesPerBlock, "RLE1 tile records live in the per-block tile scratch");

__device__ __forceinline__ int rle_w(int k) {
    const int j = k % 255;
    return j < 3 ? 1 : (j == 3 ? 2 : 0);
}
__device__ __forceinline__ int rle_G(int L) {
    const int r = L % 255;
    return 5 * (L / 255) + (r < 4 ? r : 5);
}

// Stage tile bytes [ts, te) of block B in s and find the run starts of this
// thread's 16 positions (bit q of the mask: position 16 * tid + q starts a
// run). Returns the mask; first / last are tile offsets (kRleTile / -1 when
// the thread has no start).
__device__ __forceinline__ uint32_t rle_tile_starts(const uint8_t *src, int ts, int te, uint8_t *s, int &first,
                                                    int &last) {
    const int len = te - ts;
    if (len == kRleTile && (((uintptr_t)(src + ts)) & 15) == 0) {
        reinterpret_cast<uint4 *>(s)[threadIdx.x] = __ldg(reinterpret_cast<const uint4 *>(src + ts) + threadIdx.x);
    } else {
        for (int k = threadIdx.x; k < len; k += kRleThreads) s[k] = src[ts + k];
    }
    __syncthreads();
    const int a = 16 * threadIdx.x;
    uint32_t mask = 0;
    first = kRleTile;
    last = -1;
    if (a < len) {
        int c = a > 0 ? (int)s[a - 1] : (ts > 0 ? (int)src[ts - 1] : -1);
        uint8_t v[16];
        *reinterpret_cast<uint4 *>(v) = reinterpret_cast<const uint4 *>(s)[threadIdx.x];
#pragma unroll
        for (int q = 0; q < 16; q++) {
            if (a + q < len && (int)v[q] != c) {
                mask |= 1u << q;
                first = min(first, a + q);
                last = a + q;
            }
            c = v[q];
        }
    }
    return mask;
}

// (1) aux[tile] = {first start (absolute; tile end if none), last start
//     (absolute; -1 if none), output of the positions after the first start}.
__global__ void __launch_bounds__(kRleThreads) rle1_tile_kernel(const BlockDesc *__restrict__ blocks,
                                                                int32_t *__restrict__ aux_all) {
    __shared__ __align__(16) uint8_t s[kRleTile];
    __shared__ int sh[33];
    __shared__ int sfirst, slast;
    const int b = blockIdx.y, tile = blockIdx.x;
    const BlockDesc B = blocks[b];
    const int ts = tile * kRleTile;
    if (ts >= B.len) return;
    const int te = min(B.len, ts + kRleTile);
    if (threadIdx.x == 0) { sfirst = kRleTile; slast = -1; }
    int first, last;
    const uint32_t mask = rle_tile_starts(B.src, ts, te, s, first, last);
    const int carry = block_excl_max(last, sh);
    int rs = carry, out = 0;
    const int a = 16 * threadIdx.x;
#pragma unroll
    for (int q = 0; q < 16; q++) {
        if (mask & (1u << q)) rs = a + q;
        if (rs >= 0 && a + q < te - ts) out += rle_w(a + q - rs);
    }
    int total;
    block_excl_sum<int>(out, sh, &total);
    if (first < kRleTile) atomicMin(&sfirst, first);
    if (last >= 0) atomicMax(&slast, last);
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t *aux = aux_all + ((size_t)b * kTilesPerBlock + tile) * 4;
        aux[0] = sfirst < kRleTile ? ts + sfirst : te;
        aux[1] = slast >= 0 ? ts + slast : -1;
        aux[2] = total;
    }
}

// (2) one warp per block: aux[tile][1] = run start carried into the tile,
//     aux[tile][2] = the tile's output offset; st.m = RLE1 length.
__global__ void __launch_bounds__(32) rle1_scan_kernel(const BlockDesc *__restrict__ blocks,
                                                       BlockState *__restrict__ st, int32_t *__restrict__ aux_all) {
    const int b = blockIdx.x;
    const int n = blocks[b].len;
    const int ntile = (n + kRleTile - 1) / kRleTile;
    int32_t *aux = aux_all + (size_t)b * kTilesPerBlock * 4;
    const int lane = (int)lane_id();
    int carryR = -1, carryO = 0;
    for (int base = 0; base < ntile; base += 32) {
        const int t = base + lane;
        const bool valid = t < ntile;
        const int fs = valid ? aux[t * 4 + 0] : n;
        const int ls = valid ? aux[t * 4 + 1] : -1;
        const int lo = valid ? aux[t * 4 + 2] : 0;
        const int imax = warp_incl_max(ls);
        int ex = __shfl_up_sync(LFC_FULL, imax, 1);
        if (lane == 0) ex = -1;
        const int R = max(carryR, ex);
        const int ts = t * kRleTile;
        const int pre = (valid && R >= 0) ? rle_G(fs - R) - rle_G(ts - R) : 0;
        const int out = valid ? pre + lo : 0;
        const int incl = warp_incl_sum(out);
        if (valid) {
            aux[t * 4 + 1] = R;
            aux[t * 4 + 2] = carryO + incl - out;
        }
        carryR = max(carryR, __shfl_sync(LFC_FULL, imax, 31));
        carryO += __shfl_sync(LFC_FULL, incl, 31);
    }
    if (lane == 0) st[b].m = carryO;
}

// (3) every position's output offset and bytes; the count byte of a piece
//     needs its run's end, found among the next <= 252 positions.
__global__ void __launch_bounds__(kRleThreads) rle1_write_kernel(const BlockDesc *__restrict__ blocks,
                                                                 const int32_t *__restrict__ aux_all,
                                                                 uint8_t *__restrict__ rle_all) {
    __shared__ __align__(16) uint8_t s[kRleTile];
    __shared__ uint8_t ob[kRleOutCap];
    __shared__ int sh[33];
    __shared__ int tfirst[kRleThreads];
    const int b = blockIdx.y, tile = blockIdx.x;
    const BlockDesc B = blocks[b];
    const int n = B.len, ts = tile * kRleTile;
    if (ts >= n) return;
    const int te = min(n, ts + kRleTile), len = te - ts;
    const int ntile = (n + kRleTile - 1) / kRleTile;
    const int32_t *aux = aux_all + ((size_t)b * kTilesPerBlock + tile) * 4;
    const int R = aux[1], off = aux[2];
    const int next_fs = tile + 1 < ntile ? aux[4] : n;
    int first, last;
    const uint32_t mask = rle_tile_starts(B.src, ts, te, s, first, last);
    tfirst[threadIdx.x] = first < kRleTile ? ts + first : INT_MAX;
    const int carry = block_excl_max(last >= 0 ? ts + last : -1, sh);  // also orders tfirst
    const int a = 16 * threadIdx.x;
    int rs = max(carry, R), cnt = 0;
    uint8_t w[16];
#pragma unroll
    for (int q = 0; q < 16; q++) {
        if (mask & (1u << q)) rs = ts + a + q;
        w[q] = (a + q < len) ? (uint8_t)rle_w(ts + a + q - rs) : 0;
        cnt += w[q];
    }
    int total;
    int o = block_excl_sum<int>(cnt, sh, &total);
    rs = max(carry, R);
    for (int q = 0; q < 16; q++) {
        if (mask & (1u << q)) rs = ts + a + q;
        if (!w[q]) continue;
        const uint8_t v = s[a + q];
        ob[o++] = v;
        if (w[q] == 2) {
            const int i = ts + a + q, cap = i - 3 + 255;
            int end;
            const uint32_t later = q < 15 ? (mask >> (q + 1)) : 0u;
            if (later) {
                end = i + 1 + __ffs(later) - 1;
            } else {
                end = next_fs;
                for (int tt = threadIdx.x + 1; tt < kRleThreads && ts + 16 * tt < cap; tt++)
                    if (tfirst[tt] != INT_MAX) { end = tfirst[tt]; break; }
            }
            ob[o++] = (uint8_t)(min(end, cap) - (i - 3) - 4);
        }
    }
    __syncthreads();
    uint8_t *out = rle_all + (size_t)b * kBlockCap + off;
    for (int k = threadIdx.x; k < total; k += kRleThreads) out[k] = ob[k];
}

cudaError_t launch_rle1(lfc_plan P, int nblocks, const BlockDesc *d_blocks) {
    Workspace &ws = P->ws;
    const dim3 grid(kRleMaxTiles, nblocks);
    rle1_tile_kernel<<<grid, kRleThreads, 0, P->stream>>>(d_blocks, ws.tileaux);
    rle1_scan_kernel<<<nblocks, 32, 0, P->stream>>>(d_blocks, ws.bstate, ws.tileaux);
    rle1_write_kernel<<<grid, kRleThreads, 0, P->stream>>>(d_blocks, ws.tileaux, ws.rle);
    count_launches(P, 3);
    return cudaGetLastError();
}

// ------------------------------------------------------------ sort keys
template <int MODE>
__device__ __forceinline__ int sort_count(const BlockState &s, int h) {
    if (MODE == 0) return s.m;
    return h < s.m ? s.n_act : 0;
}

template <int MODE>
__device__ __forceinline__ int round_h(const int32_t *rs) { return MODE == 0 ? 0 : rs[2]; }

// Phase 1 keys: K[v] = bytes v .. v + 7 (cyclic) big-endian, element v.
// Phase 1 sorts the first kPhase1Bytes bytes of every rotation; they sit in
// the top bytes of the 64-bit key, so passes 8 - kPhase1Bytes .. 7 carry them.
constexpr int kPhase1Bytes = LFC_PHASE1_BYTES;

__global__ void __launch_bounds__(kSortThreads) key8_kernel(const BlockState *__restrict__ st,
                                                            const uint8_t *__restrict__ rle_all,
                                                            uint64_t *__restrict__ K_all, int32_t *__restrict__ V_all) {
    __shared__ uint8_t sb[kTile + 8];
    const int b = blockIdx.y, tile = blockIdx.x;
    const int m = st[b].m;
    const int t0 = tile * kTile;
    if (t0 >= m) return;
    const int cnt = min(kTile, m - t0);
    const uint8_t *rle = rle_all + (size_t)b * kBlockCap;
    for (int i = threadIdx.x; i < cnt + 7; i += kSortThreads) sb[i] = rle[(t0 + i) % m];
    __syncthreads();
    uint64_t *K = K_all + (size_t)b * kBlockCap;
    int32_t *V = V_all + (size_t)b * kBlockCap;
    for (int r = 0; r < kPerThread; r++) {
        const int kl = r * kSortThreads + threadIdx.x;
        if (kl >= cnt) break;
        uint64_t key = 0;
#pragma unroll
        for (int q = 0; q < kPhase1Bytes; q++) key = (key << 8) | sb[kl + q];
        K[t0 + kl] = key << (8 * (8 - kPhase1Bytes));
        V[t0 + kl] = t0 + kl;
    }
}

// Round words of the tied elements: rank[v] << 40 | rank[(v + h) mod m] << 20 | v.
constexpr uint64_t kElemMask = (1u << 20) - 1u;

__global__ void __launch_bounds__(kSortThreads) key40_kernel(const int32_t *__restrict__ rs, const BlockState *__restrict__ st,
                                                             const int32_t *__restrict__ V_all, const int32_t *__restrict__ rank_all,
                                                             uint64_t *__restrict__ K_all) {
    const int b = blockIdx.y, tile = blockIdx.x;
    const int h = rs[2];
    const BlockState s = st[b];
    const int n = sort_count<1>(s, h);
    const size_t bo = (size_t)b * kBlockCap;
    for (int r = 0; r < kPerThread; r++) {
        const int k = tile * kTile + r * kSortThreads + threadIdx.x;
        if (k >= n) break;
        const int v = V_all[bo + k];
        int j = v + h;
        if (j >= s.m) j -= s.m;
        K_all[bo + k] = ((uint64_t)(uint32_t)rank_all[bo + v] << 40) | ((uint64_t)(uint32_t)rank_all[bo + j] << 20) |
                        (uint64_t)(uint32_t)v;
    }
}

// Digit position of a pass: phase 1 sorts all 64 key bits, a round bits 20..59.
template <int MODE>
__device__ __forceinline__ int digit_shift(int pass) { return (MODE == 0 ? 0 : 20) + 8 * pass; }

// Per-tile digit histogram, stored digit-major: cnt[b][digit][tile]. A warp
// whose 32 digits agree adds them with one atomic (long equal runs are the
// norm in these streams).
// Round state in device memory: rs[0] tied elements after the round, rs[1]
// their per-block maximum, rs[2] the shift h, rs[3] the round number.
template <int MODE>
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(int pass, const int32_t *__restrict__ rs, const BlockState *__restrict__ st,
                                                                  const uint64_t *__restrict__ K_all, uint32_t *__restrict__ cnt_all) {
    constexpr int NW = kSortThreads / 32;
    __shared__ uint32_t hst[NW][256];
    const int b = blockIdx.y, tile = blockIdx.x;
    const int h = round_h<MODE>(rs);
    const int n = sort_count<MODE>(st[b], h);
    if (tile * kTile >= n) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < NW * 256; i += kSortThreads) (&hst[0][0])[i] = 0;
    __syncthreads();
    const uint64_t *K = K_all + (size_t)b * kBlockCap;
    const int shift = digit_shift<MODE>(pass);
    uint32_t dg[kPerThread];
#pragma unroll
    for (int r = 0; r < kPerThread; r++) {  // all loads in flight first
        const int k = tile * kTile + w * 512 + r * 32 + lane;
        dg[r] = k < n ? (uint32_t)(K[k] >> shift) & 255u : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int r = 0; r < kPerThread; r++) {
        const uint32_t d = dg[r];
        const uint32_t d0 = __shfl_sync(LFC_FULL, d, 0);
        if (__all_sync(LFC_FULL, d == d0)) {
            if (lane == 0 && d0 != 0xFFFFFFFFu) atomicAdd(&hst[w][d0], 32u);
        } else if (d != 0xFFFFFFFFu) {
            atomicAdd(&hst[w][d], 1u);
        }
    }
    __syncthreads();
    uint32_t c = 0;
    for (int i = 0; i < NW; i++) c += hst[i][threadIdx.x];
    cnt_all[((size_t)b * 256 + threadIdx.x) * kTilesPerBlock + tile] = c;
}

// Exclusive scan of a block's counts in (digit, tile) order, in place.
template <int MODE>
__global__ void __launch_bounds__(1024) radix_scan_kernel(const int32_t *__restrict__ rs, const BlockState *__restrict__ st, uint32_t *__restrict__ cnt_all) {
    __shared__ uint32_t sh[33];
    const int b = blockIdx.x;
    const int h = round_h<MODE>(rs);
    const int n = sort_count<MODE>(st[b], h);
    if (n == 0) return;
    const int nt = (n + kTile - 1) / kTile;
    const int total = 256 * nt;
    uint32_t *cnt = cnt_all + (size_t)b * 256 * kTilesPerBlock;
    const int per = (total + blockDim.x - 1) / blockDim.x;
    const int a = min(total, (int)threadIdx.x * per), e = min(total, a + per);
    const int d0 = a / nt, t0 = a - d0 * nt;  // (digit, tile) of the first entry
    // batches of independent loads: a thread's entries cost a few round trips
    constexpr int kBatch = 16;
    uint32_t sum = 0;
    for (int q0 = a, d = d0, t = t0; q0 < e; q0 += kBatch) {
        uint32_t v[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; j++) {
            v[j] = q0 + j < e ? cnt[d * kTilesPerBlock + t] : 0u;
            if (++t == nt) { t = 0; d++; }
        }
#pragma unroll
        for (int j = 0; j < kBatch; j++) sum += v[j];
    }
    uint32_t off = block_excl_sum<uint32_t>(sum, sh, nullptr);
    for (int q0 = a, d = d0, t = t0; q0 < e; q0 += kBatch) {
        uint32_t v[kBatch];
        int dj[kBatch], tj[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; j++) {
            dj[j] = d;
            tj[j] = t;
            v[j] = q0 + j < e ? cnt[d * kTilesPerBlock + t] : 0u;
            if (++t == nt) { t = 0; d++; }
        }
#pragma unroll
        for (int j = 0; j < kBatch; j++) {
            if (q0 + j < e) cnt[dj[j] * kTilesPerBlock + tj[j]] = off;
            off += v[j];
        }
    }
}

// Stable scatter of (key, element) pairs: warp w owns elements
// [w*512, (w+1)*512) of the tile, taken 32 at a time in order; equal digits
// are ranked with __match_any_sync and a per-warp running count. The tile is
// placed in shared memory in digit order, then each digit's run is written
// to its global offset with consecutive threads on consecutive addresses.
constexpr size_t kScatterSmem = (size_t)kTile * 12 + (size_t)(kSortThreads / 32) * 256 * 4 + 2 * 256 * 4;
// MODE 1 moves the words alone (Vin / Vout unused)
constexpr size_t kScatterSmem1 = (size_t)kTile * 8 + (size_t)(kSortThreads / 32) * 256 * 4 + 2 * 256 * 4;

template <int MODE>
__global__ void __launch_bounds__(kSortThreads, 3) radix_scatter_kernel(int pass, const int32_t *__restrict__ rs, const BlockState *__restrict__ st,
                                                                     const uint64_t *__restrict__ Kin_all, const int32_t *__restrict__ Vin_all,
                                                                     uint64_t *__restrict__ Kout_all, int32_t *__restrict__ Vout_all,
                                                                     const uint32_t *__restrict__ cnt_all) {
    constexpr int NW = kSortThreads / 32;
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t *sK = reinterpret_cast<uint64_t *>(smem);           // [kTile]
    int32_t *sV = reinterpret_cast<int32_t *>(sK + kTile);        // [kTile], MODE 0
    uint32_t *wcnt = reinterpret_cast<uint32_t *>(MODE == 0 ? reinterpret_cast<uint8_t *>(sV + kTile)
                                                            : reinterpret_cast<uint8_t *>(sK + kTile));  // [NW][256]
    uint32_t *loff = wcnt + NW * 256;                             // [256] tile-local start of a digit
    uint32_t *gbase = loff + 256;                                 // [256] global start of the tile's run
    __shared__ uint32_t sh[33];
    const int b = blockIdx.y, tile = blockIdx.x;
    const int h = round_h<MODE>(rs);
    const int n = sort_count<MODE>(st[b], h);
    if (tile * kTile >= n) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int shift = digit_shift<MODE>(pass);
    for (int i = threadIdx.x; i < NW * 256; i += kSortThreads) wcnt[i] = 0;
    gbase[threadIdx.x] = cnt_all[((size_t)b * 256 + threadIdx.x) * kTilesPerBlock + tile];
    __syncthreads();
    const size_t bo = (size_t)b * kBlockCap;
    const uint64_t *Kin = Kin_all + bo;
    const int32_t *Vin = Vin_all + bo;
    uint64_t keys[kPerThread];
    int32_t vals[kPerThread];
    uint32_t rnk[kPerThread];
    const uint32_t lt = lanemask_lt(), gt = lanemask_gt();
#pragma unroll
    for (int r = 0; r < kPerThread; r++) {
        const int k = tile * kTile + w * 512 + r * 32 + lane;
        const bool ok = k < n;
        keys[r] = ok ? Kin[k] : 0;
        vals[r] = (MODE == 0 && ok) ? Vin[k] : 0;
        const uint32_t d = (uint32_t)(keys[r] >> shift) & 255u;
        const uint32_t mm = __match_any_sync(LFC_FULL, ok ? d : 256u + lane);
        uint32_t before = 0;
        if (ok) before = wcnt[w * 256 + d];
        __syncwarp();
        if (ok && (mm & gt) == 0) wcnt[w * 256 + d] = before + __popc(mm);
        __syncwarp();
        rnk[r] = ok ? before + __popc(mm & lt) : 0xFFFFFFFFu;
    }
    __syncthreads();
    {   // per digit: exclusive prefix over warps, then over digits
        const int d = threadIdx.x;
        uint32_t acc = 0;
        for (int ww = 0; ww < NW; ww++) {
            const uint32_t c = wcnt[ww * 256 + d];
            wcnt[ww * 256 + d] = acc;
            acc += c;
        }
        loff[d] = block_excl_sum<uint32_t>(acc, sh, nullptr);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPerThread; r++) {
        if (rnk[r] == 0xFFFFFFFFu) continue;
        const uint32_t d = (uint32_t)(keys[r] >> shift) & 255u;
        const uint32_t pos = loff[d] + wcnt[w * 256 + d] + rnk[r];
        sK[pos] = keys[r];
        if (MODE == 0) sV[pos] = vals[r];
    }
    __syncthreads();
    const int cnt = min(kTile, n - tile * kTile);
    uint64_t *Kout = Kout_all + bo;
    int32_t *Vout = Vout_all + bo;
#pragma unroll 4
    for (int r = 0; r < kPerThread; r++) {
        const int j = r * kSortThreads + threadIdx.x;
        if (j < cnt) {
            const uint64_t key = sK[j];
            const uint32_t d = (uint32_t)(key >> shift) & 255u;
            const uint32_t g = gbase[d] + ((uint32_t)j - loff[d]);
            Kout[g] = key;
            if (MODE == 0) Vout[g] = sV[j];
        }
    }
}

// ---------------------------------------------------------- group heads
// Head flags come from neighbouring keys of the sorted (key, element) list:
// the 8-byte prefixes after phase 1, the 40-bit round keys after a round.
// Pass A: per tile, the largest head position and the number of elements
// that stay tied. Head flags go to flags[] for pass B.
template <int MODE>
__global__ void __launch_bounds__(kSortThreads) heads_tile_kernel(const int32_t *__restrict__ rs, const BlockState *__restrict__ st,
                                                                  const uint64_t *__restrict__ keys_all, const int32_t *__restrict__ actA,
                                                                  const int32_t *__restrict__ actB,
                                                                  uint8_t *__restrict__ flags_all, int32_t *__restrict__ aux_all) {
    const int b = blockIdx.y, tile = blockIdx.x;
    const int h = round_h<MODE>(rs);
    const BlockState s = st[b];
    const int n = sort_count<MODE>(s, h);
    if (tile * kTile >= n) return;
    const uint64_t *K = keys_all + (size_t)b * kBlockCap;
    const int32_t *act = ((MODE == 1 && (rs[3] & 1)) ? actB : actA) + (size_t)b * kBlockCap;
    uint8_t *flags = flags_all + (size_t)b * kBlockCap;
    const int k0 = tile * kTile + threadIdx.x * kPerThread;
    int hmax = -1, tied = 0;
    const int ks = MODE == 0 ? 0 : 20;  // round words carry the element below the key
    if (k0 + kPerThread <= n) {  // full run: 16-byte loads of the keys, one 16-byte store of the flags
        uint64_t kk[kPerThread];
        const ulonglong2 *K2 = reinterpret_cast<const ulonglong2 *>(K + k0);
#pragma unroll
        for (int q = 0; q < kPerThread / 2; q++) {
            const ulonglong2 v = K2[q];
            kk[2 * q] = v.x >> ks;
            kk[2 * q + 1] = v.y >> ks;
        }
        const bool last_head = k0 + kPerThread >= n || (K[k0 + kPerThread] >> ks) != kk[kPerThread - 1];
        bool curhead = (k0 == 0) || kk[0] != (K[k0 - (k0 > 0)] >> ks);
        uint32_t fl[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int q = 0; q < kPerThread; q++) {
            const bool nexthead = q + 1 < kPerThread ? kk[q + 1] != kk[q] : last_head;
            if (curhead) {
                fl[q >> 2] |= 1u << (8 * (q & 3));
                hmax = MODE == 0 ? k0 + q : act[k0 + q];
            }
            tied += !(curhead && nexthead);
            curhead = nexthead;
        }
        *reinterpret_cast<uint4 *>(flags + k0) = make_uint4(fl[0], fl[1], fl[2], fl[3]);
    } else if (k0 < n) {
        const int k1 = min(n, k0 + kPerThread);
        uint64_t prevk = k0 > 0 ? K[k0 - 1] >> ks : 0;
        uint64_t cur = K[k0] >> ks;
        bool curhead = (k0 == 0) || cur != prevk;
        for (int k = k0; k < k1; k++) {
            bool nexthead = true;
            uint64_t nk = 0;
            if (k + 1 < n) {
                nk = K[k + 1] >> ks;
                nexthead = nk != cur;
            }
            flags[k] = (uint8_t)curhead;
            if (curhead) hmax = MODE == 0 ? k : act[k];
            tied += !(curhead && nexthead);
            cur = nk;
            curhead = nexthead;
        }
    }
    int mine = hmax;  // last head position among this thread's elements
    for (int o = 16; o > 0; o >>= 1) mine = max(mine, __shfl_xor_sync(LFC_FULL, mine, o));
    for (int o = 16; o > 0; o >>= 1) tied += __shfl_xor_sync(LFC_FULL, tied, o);
    __shared__ int32_t wm[kSortThreads / 32], wt[kSortThreads / 32];
    if ((threadIdx.x & 31) == 0) { wm[threadIdx.x >> 5] = mine; wt[threadIdx.x >> 5] = tied; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int mx = -1, tt = 0;
        for (int i = 0; i < kSortThreads / 32; i++) { mx = max(mx, wm[i]); tt += wt[i]; }
        int32_t *aux = aux_all + ((size_t)b * kTilesPerBlock + tile) * 4;
        aux[0] = mx;
        aux[1] = tt;
    }
}

// Pass across tiles of a block: exclusive max of head positions, exclusive
// sum of tied counts, total tied count of the block.
template <int MODE>
__global__ void __launch_bounds__(256) heads_scan_kernel(int32_t *__restrict__ rs, BlockState *__restrict__ st, int32_t *__restrict__ aux_all) {
    __shared__ int32_t shm[33];
    __shared__ int32_t shs[33];
    const int b = blockIdx.x;
    const int h = round_h<MODE>(rs);
    int32_t *counters = rs;
    const int n = sort_count<MODE>(st[b], h);
    int32_t *aux = aux_all + (size_t)b * kTilesPerBlock * 4;
    const int nt = (n + kTile - 1) / kTile;
    // nt <= 220 < 256: one tile per thread
    const int t = threadIdx.x;
    const int mx = t < nt ? aux[t * 4 + 0] : -1;
    const int cn = t < nt ? aux[t * 4 + 1] : 0;
    const int exm = block_excl_max(mx, shm);
    int total;
    const int exs = block_excl_sum<int>(cn, shs, &total);
    if (t < nt) { aux[t * 4 + 2] = exm; aux[t * 4 + 3] = exs; }
    if (t == 0) {
        st[b].n_act_next = total;
        if (total) { atomicAdd(&counters[0], total); atomicMax(&counters[1], total); }
    }
}

// Pass B: rank[v] = head position of v's group; the suffix array takes the
// sorted tied elements (MODE 1); elements still tied are compacted into the
// next round's lists.
template <int MODE>
__global__ void __launch_bounds__(kSortThreads) heads_apply_kernel(const int32_t *__restrict__ rs, const BlockState *__restrict__ st,
                                                                   const int32_t *__restrict__ sorted_all, const uint64_t *__restrict__ words_all,
                                                                   int32_t *__restrict__ actA,
                                                                   int32_t *__restrict__ actB,
                                                                   const uint8_t *__restrict__ flags_all, const int32_t *__restrict__ aux_all,
                                                                   int32_t *__restrict__ rank_all, int32_t *__restrict__ sa_all,
                                                                   int32_t *__restrict__ val_out_all) {
    __shared__ int32_t shm[33];
    __shared__ int32_t shs[33];
    const int b = blockIdx.y, tile = blockIdx.x;
    const int h = round_h<MODE>(rs);
    // round r reads list A (r even) or B (r odd) and writes the other; the
    // initial pass (MODE 0) writes A, which round 0 reads
    const bool odd = MODE == 1 && (rs[3] & 1);
    const int32_t *act_all = odd ? actB : actA;
    int32_t *act_out_all = MODE == 0 ? actA : (odd ? actA : actB);
    const BlockState s = st[b];
    const int n = sort_count<MODE>(s, h);
    if (tile * kTile >= n) return;
    const size_t bo = (size_t)b * kBlockCap;
    const int32_t *sorted = sorted_all + bo;   // MODE 0: the suffix array
    const uint64_t *words = words_all + bo;    // MODE 1: sorted round words
    const int32_t *act = act_all + bo;
    const uint8_t *flags = flags_all + bo;
    const int32_t *aux = aux_all + ((size_t)b * kTilesPerBlock + tile) * 4;
    int32_t *rank = rank_all + bo;
    int32_t *sa = sa_all + bo;
    int32_t *act_out = act_out_all + bo;
    int32_t *val_out = val_out_all + bo;
    const int k0 = tile * kTile + threadIdx.x * kPerThread;
    const int k1 = min(n, k0 + kPerThread);
    int mine = -1, tied = 0;
    // a full run loads flags, positions and elements with 16-byte loads; the
    // block scans are reached by every thread
    const bool full = k0 + kPerThread <= n;
    uint32_t fw[4] = {0u, 0u, 0u, 0u};
    bool last_next = true;
    int32_t pv[kPerThread];
    if (full) {
        const uint4 f4 = *reinterpret_cast<const uint4 *>(flags + k0);
        fw[0] = f4.x; fw[1] = f4.y; fw[2] = f4.z; fw[3] = f4.w;
        last_next = k0 + kPerThread >= n || flags[k0 + kPerThread];
#pragma unroll
        for (int q = 0; q < kPerThread; q += 4) {
            if (MODE == 1) {
                const int4 a4 = *reinterpret_cast<const int4 *>(act + k0 + q);
                pv[q] = a4.x; pv[q + 1] = a4.y; pv[q + 2] = a4.z; pv[q + 3] = a4.w;
            } else {
                pv[q] = k0 + q; pv[q + 1] = k0 + q + 1; pv[q + 2] = k0 + q + 2; pv[q + 3] = k0 + q + 3;
            }
        }
#pragma unroll
        for (int q = 0; q < kPerThread; q++) {
            const bool hd = (fw[q >> 2] >> (8 * (q & 3))) & 1u;
            const bool nh = q + 1 < kPerThread ? ((fw[(q + 1) >> 2] >> (8 * ((q + 1) & 3))) & 1u) : last_next;
            if (hd) mine = pv[q];
            tied += !(hd && nh);
        }
    } else {
        for (int k = k0; k < k1; k++) {
            const bool hd = flags[k];
            const bool nh = (k + 1 >= n) || flags[k + 1];
            if (hd) mine = MODE == 0 ? k : act[k];
            tied += !(hd && nh);
        }
    }
    int carry = block_excl_max(mine, shm);
    carry = max(carry, aux[2]);
    int off = block_excl_sum<int>(tied, shs, nullptr) + aux[3];
    if (full) {
        int32_t vv[kPerThread];
#pragma unroll
        for (int q = 0; q < kPerThread; q += 4) {
            if (MODE == 0) {
                const int4 s4 = *reinterpret_cast<const int4 *>(sorted + k0 + q);
                vv[q] = s4.x; vv[q + 1] = s4.y; vv[q + 2] = s4.z; vv[q + 3] = s4.w;
            } else {
                const ulonglong2 w0 = *reinterpret_cast<const ulonglong2 *>(words + k0 + q);
                const ulonglong2 w1 = *reinterpret_cast<const ulonglong2 *>(words + k0 + q + 2);
                vv[q] = (int32_t)(w0.x & kElemMask); vv[q + 1] = (int32_t)(w0.y & kElemMask);
                vv[q + 2] = (int32_t)(w1.x & kElemMask); vv[q + 3] = (int32_t)(w1.y & kElemMask);
            }
        }
#pragma unroll
        for (int q = 0; q < kPerThread; q++) {
            const bool hd = (fw[q >> 2] >> (8 * (q & 3))) & 1u;
            const bool nh = q + 1 < kPerThread ? ((fw[(q + 1) >> 2] >> (8 * ((q + 1) & 3))) & 1u) : last_next;
            const int pos = pv[q];
            if (hd) carry = pos;
            const int32_t v = vv[q];
            rank[v] = carry;
            if (MODE == 1 || sorted != sa) sa[pos] = v;
            if (!(hd && nh)) {
                act_out[off] = pos;
                val_out[off] = v;
                off++;
            }
        }
        return;
    }
    for (int k = k0; k < k1; k++) {
        const bool hd = flags[k];
        const bool nh = (k + 1 >= n) || flags[k + 1];
        const int pos = MODE == 0 ? k : act[k];
        if (hd) carry = pos;
        const int32_t v = MODE == 0 ? sorted[k] : (int32_t)(words[k] & kElemMask);
        rank[v] = carry;
        if (MODE == 1 || sorted != sa) sa[pos] = v;
        if (!(hd && nh)) {
            act_out[off] = pos;
            val_out[off] = v;
            off++;
        }
    }
}

__global__ void commit_round_kernel(BlockState *st, int nblocks) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nblocks) { st[b].n_act = st[b].n_act_next; st[b].n_act_next = 0; }
}

__global__ void round_start_kernel(int32_t *rs, int first) {
    rs[0] = 0;
    rs[1] = 0;
    if (first) { rs[2] = kPhase1Bytes; rs[3] = 0; }
}

// End of a doubling round: double h; inside a graph, continue the WHILE node
// while tied elements remain and h is below the largest block length.
__global__ void round_end_kernel(int32_t *rs, int max_m, cudaGraphConditionalHandle cond, int set_cond) {
    rs[2] *= 2;
    rs[3] += 1;
    if (set_cond) cudaGraphSetConditional(cond, (rs[0] > 0 && rs[2] < max_m) ? 1u : 0u);
}

// L[j] = block[(SA[j] - 1) mod m]; origPtr = j with SA[j] = 0; bytes in use.
// Each CTA also writes the MTF summary of its 4096-byte segment of L: the
// distinct bytes ordered by last occurrence, latest first. Thread = 16
// consecutive positions; the last position of each byte value comes from one
// shared-memory max per distinct value of a thread's run; each value is then
// marked at its last position and the marks are compacted from the top.
__global__ void __launch_bounds__(kSortThreads) bwt_output_kernel(BlockState *__restrict__ st, const int32_t *__restrict__ sa_all,
                                                                  const uint8_t *__restrict__ rle_all, uint8_t *__restrict__ L_all,
                                                                  uint8_t *__restrict__ rec_all, int32_t *__restrict__ reclen_all) {
    __shared__ int32_t lastpos[256];
    __shared__ uint16_t mark[kTile];  // value + 1 at its last position, 0 elsewhere
    __shared__ int sh[33];
    const int b = blockIdx.y, tile = blockIdx.x;
    const int m = st[b].m;
    if (tile * kTile >= m) return;
    lastpos[threadIdx.x] = -1;
    for (int i = threadIdx.x; i < kTile; i += kSortThreads) mark[i] = 0;
    __syncthreads();
    const size_t bo = (size_t)b * kBlockCap;
    const int jl = (int)threadIdx.x * kPerThread;  // tile-local start of the thread's run
    const int j0 = tile * kTile + jl;
    uint8_t c[kPerThread];
    int32_t sv[kPerThread];
    if (j0 + kPerThread <= m) {  // full run: the suffix array by 16-byte loads
#pragma unroll
        for (int q = 0; q < kPerThread; q += 4) {
            const int4 s4 = *reinterpret_cast<const int4 *>(sa_all + bo + j0 + q);
            sv[q] = s4.x; sv[q + 1] = s4.y; sv[q + 2] = s4.z; sv[q + 3] = s4.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < kPerThread; q++) sv[q] = j0 + q < m ? sa_all[bo + j0 + q] : -1;
    }
#pragma unroll
    for (int q = 0; q < kPerThread; q++) {
        const int v = sv[q];
        c[q] = 0;
        if (v >= 0) {
            c[q] = rle_all[bo + (v == 0 ? m - 1 : v - 1)];
            if (v == 0) st[b].orig_ptr = j0 + q;
        }
    }
    if (j0 + kPerThread <= m) {
        uint32_t pk[4];
#pragma unroll
        for (int w = 0; w < 4; w++)
            pk[w] = (uint32_t)c[4 * w] | ((uint32_t)c[4 * w + 1] << 8) | ((uint32_t)c[4 * w + 2] << 16) |
                    ((uint32_t)c[4 * w + 3] << 24);
        *reinterpret_cast<uint4 *>(L_all + bo + j0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    } else {
#pragma unroll
        for (int q = 0; q < kPerThread; q++)
            if (j0 + q < m) L_all[bo + j0 + q] = c[q];
    }
#pragma unroll
    for (int q = kPerThread - 1; q >= 0; q--) {  // last occurrence in the run first
        if (j0 + q >= m) continue;
        bool seen = false;
#pragma unroll
        for (int r = q + 1; r < kPerThread; r++) seen |= (j0 + r < m) && c[r] == c[q];
        if (!seen) atomicMax(&lastpos[c[q]], jl + q);
    }
    __syncthreads();
    const int x = threadIdx.x;
    const int lp = lastpos[x];
    if (lp >= 0) mark[lp] = (uint16_t)(x + 1);
    const uint32_t present = __ballot_sync(LFC_FULL, lp >= 0);  // values 32 w .. 32 w + 31
    if ((threadIdx.x & 31) == 0 && present) atomicOr(&st[b].in_use[threadIdx.x >> 5], present);
    __syncthreads();
    // compaction, highest positions first: thread t takes positions 4095 - 16 t - q
    const int top = kTile - 1 - jl;
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < kPerThread; q++) cnt += mark[top - q] != 0;
    int total;
    int o = block_excl_sum<int>(cnt, sh, &total);
    uint8_t *rec = rec_all + ((size_t)b * kTilesPerBlock + tile) * 256;
#pragma unroll
    for (int q = 0; q < kPerThread; q++) {
        const uint16_t mv = mark[top - q];
        if (mv) rec[o++] = (uint8_t)(mv - 1);
    }
    if (threadIdx.x == 0) reclen_all[(size_t)b * kTilesPerBlock + tile] = total;
}

template <int MODE>
static void radix_pass(lfc_plan P, cudaStream_t st, int nblocks, int tiles, int pass, const uint64_t *kin, const int32_t *vin,
                       uint64_t *kout, int32_t *vout) {
    Workspace &ws = P->ws;
    dim3 grid(tiles, nblocks);
    radix_hist_kernel<MODE><<<grid, kSortThreads, 0, st>>>(pass, ws.act_total, ws.bstate, kin, ws.tilecnt);
    radix_scan_kernel<MODE><<<nblocks, 1024, 0, st>>>(ws.act_total, ws.bstate, ws.tilecnt);
    radix_scatter_kernel<MODE><<<grid, kSortThreads, MODE == 0 ? kScatterSmem : kScatterSmem1, st>>>(
        pass, ws.act_total, ws.bstate, kin, vin, kout, vout, ws.tilecnt);
    count_launches(P, 3);
}

// One prefix-doubling round over the tied elements (h and the parity of the
// active lists come from the round state in device memory).
static void bwt_round(lfc_plan P, cudaStream_t st, int nblocks, int tiles, int max_m, cudaGraphConditionalHandle cond,
                      int set_cond) {
    Workspace &ws = P->ws;
    round_start_kernel<<<1, 1, 0, st>>>(ws.act_total, 0);
    dim3 g1(tiles, nblocks);
    key40_kernel<<<g1, kSortThreads, 0, st>>>(ws.act_total, ws.bstate, ws.val, ws.rank, ws.keys);
    // 5 LSD passes over bits 20..59 of the words: keys -> keys2 -> ... -> keys2
    for (int pass = 0; pass < 5; pass++) {
        if (pass & 1) radix_pass<1>(P, st, nblocks, tiles, pass, ws.keys2, nullptr, ws.keys, nullptr);
        else radix_pass<1>(P, st, nblocks, tiles, pass, ws.keys, nullptr, ws.keys2, nullptr);
    }
    heads_tile_kernel<1><<<g1, kSortThreads, 0, st>>>(ws.act_total, ws.bstate, ws.keys2, ws.act, ws.act2, ws.bwt,
                                                      ws.tileaux);
    heads_scan_kernel<1><<<nblocks, 256, 0, st>>>(ws.act_total, ws.bstate, ws.tileaux);
    heads_apply_kernel<1><<<g1, kSortThreads, 0, st>>>(ws.act_total, ws.bstate, nullptr, ws.keys2, ws.act, ws.act2,
                                                       ws.bwt, ws.tileaux, ws.rank, ws.sa, ws.val);
    commit_round_kernel<<<(nblocks + 255) / 256, 256, 0, st>>>(ws.bstate, nblocks);
    round_end_kernel<<<1, 1, 0, st>>>(ws.act_total, max_m, cond, set_cond);
    count_launches(P, 7);
}

cudaError_t launch_bwt(lfc_plan P, int nblocks, int max_m) {
    Workspace &ws = P->ws;
    cudaStream_t s = P->stream;
    cudaError_t e;
    const int tiles = (max_m + kTile - 1) / kTile;
    if (tiles == 0) return cudaSuccess;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    const bool graph = cap == cudaStreamCaptureStatusActive;
    e = cudaFuncSetAttribute(radix_scatter_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(radix_scatter_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem1);
    if (e != cudaSuccess) return e;
    // phase 1: prefix keys, then 8 LSD passes (keys, sa) -> (keys2, sa2) -> ... -> (keys, sa)
    stage_begin(P, LFC_STAGE_BWT_SORT8);
    dim3 grid(tiles, nblocks);
    key8_kernel<<<grid, kSortThreads, 0, s>>>(ws.bstate, ws.rle, ws.keys, ws.sa);
    count_launches(P, 1);
    uint64_t *kin = ws.keys, *kout = ws.keys2;
    int32_t *vin = ws.sa, *vout = ws.sa2;
    for (int pass = 8 - kPhase1Bytes; pass < 8; pass++) {
        radix_pass<0>(P, s, nblocks, tiles, pass, kin, vin, kout, vout);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    stage_end(P, LFC_STAGE_BWT_SORT8);  // sorted keys / suffix array now in kin / vin
    stage_begin(P, LFC_STAGE_BWT_REFINE);
    round_start_kernel<<<1, 1, 0, s>>>(ws.act_total, 1);
    heads_tile_kernel<0><<<grid, kSortThreads, 0, s>>>(ws.act_total, ws.bstate, kin, ws.sa, ws.sa, ws.bwt, ws.tileaux);
    heads_scan_kernel<0><<<nblocks, 256, 0, s>>>(ws.act_total, ws.bstate, ws.tileaux);
    heads_apply_kernel<0><<<grid, kSortThreads, 0, s>>>(ws.act_total, ws.bstate, vin, nullptr, ws.act, ws.act2,
                                                        ws.bwt, ws.tileaux, ws.rank, ws.sa, ws.val);
    commit_round_kernel<<<(nblocks + 255) / 256, 256, 0, s>>>(ws.bstate, nblocks);
    count_launches(P, 5);
    P->bwt_calls++;
    if (graph) {
        // rounds as a WHILE node: the body is one round, its last kernel
        // decides whether another round runs
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *edata = nullptr;
        size_t ndeps = 0;
        cudaGraph_t cg = nullptr;
        unsigned long long cid = 0;
        e = cudaStreamGetCaptureInfo(s, &cap, &cid, &cg, &deps, &edata, &ndeps);
        if (e != cudaSuccess) return e;
        cudaGraphConditionalHandle cond;
        e = cudaGraphConditionalHandleCreate(&cond, cg, 1, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) return e;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        e = cudaGraphAddNode(&node, cg, deps, edata, ndeps, &np);
        if (e != cudaSuccess) return e;
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(P->aux_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return e;
        bwt_round(P, P->aux_stream, nblocks, kTilesPerBlock, max_m, cond, 1);
        e = cudaStreamEndCapture(P->aux_stream, &body);
        if (e != cudaSuccess) return e;
        e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e != cudaSuccess) return e;
    } else {
        e = cudaMemcpyAsync(ws.h_act_total, ws.act_total, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        int round = 0;
        for (int h = kPhase1Bytes; ws.h_act_total[0] > 0 && h < max_m; h *= 2, round++) {
            P->bwt_rounds++;
            P->bwt_tied_total += ws.h_act_total[0];
            if (round < 32) P->bwt_round_tied[round] += ws.h_act_total[0];
            const int t1 = (ws.h_act_total[1] + kTile - 1) / kTile;
            bwt_round(P, s, nblocks, t1, max_m, cudaGraphConditionalHandle{}, 0);
            e = cudaMemcpyAsync(ws.h_act_total, ws.act_total, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return e;
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
        }
    }
    stage_end(P, LFC_STAGE_BWT_REFINE);
    stage_begin(P, LFC_STAGE_BWT_OUT);
    bwt_output_kernel<<<grid, kSortThreads, 0, s>>>(ws.bstate, ws.sa, ws.rle, ws.bwt, ws.mtfrec, ws.mtfreclen);
    stage_end(P, LFC_STAGE_BWT_OUT);
    count_launches(P, 1);
    return cudaGetLastError();
}

}  // namespace lfc

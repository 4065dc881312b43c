// bwt.cu -- RLE1 and the Burrows-Wheeler transform of every bzip2 block
// (Sec. 2.1.3 codes the chosen stream with bzip2; the block format is the
// public bzip2 format).
//
// BWT = sort of all cyclic rotations, ties between identical rotations by
// start index. Two phases over all blocks of a pass at once. Every element
// carries its sort key. A radix pass is one persistent kernel whose CTAs
// take 4096-element tiles from a device work queue, tile-major over the
// blocks so that a block has only a few tiles in flight: a CTA reads its tile's
// (key, element) pairs coalesced, ranks them by digit in shared memory,
// publishes the tile's digit counts and adds up the counts of the block's
// earlier tiles as they are published (decoupled look-back: a tile only waits
// on tiles taken from the queue before it, every wait bounded by a cycle
// budget), then writes each digit's run of the tile contiguously. The
// block's digit totals for every pass come from the kernel that builds the
// keys, so a pass needs no separate histogram or scan launch.
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
#include <algorithm>
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

// Sort state in device memory (rs): tied elements after a round, their
// per-block maximum, the shift h, the round number; the abort word (nonzero
// once a bounded wait has given up in this suffix sort: every later sort
// kernel returns at once), the fault-injection word (test hook), the two work
// queues of the radix passes (by pass parity), the work items of the current
// pass, the sticky status (kept until the host reads it), and from
// kRsTileOff on the per-block prefix of tile counts (nblocks + 1 entries).
enum : int {
    kRsTied = 0, kRsTiedMax = 1, kRsH = 2, kRsRound = 3, kRsAbort = 4, kRsFault = kSortFaultWord, kRsQueue = 6,
    kRsItems = 8, kRsSticky = kSortStickyWord, kRsTileOff = 16
};
static_assert(kRsTileOff == kSortCtlHead, "sort control layout");

// Look-back status word of one digit of one tile: bits 30-31 a flag, bits
// 0-29 a count (at most kBlockCap < 2^30).
constexpr uint32_t kLbAgg = 1u << 30;   // the tile's own count
constexpr uint32_t kLbIncl = 2u << 30;  // count of this tile and every earlier tile of the block
constexpr uint32_t kLbCount = (1u << 30) - 1u;
constexpr size_t kLbBlockWords = (size_t)kTilesPerBlock * 256;  // one block's words in one status array
constexpr int kSweepPasses = 8;  // digit-histogram rows per block (phase 1: 8 passes, a round: 5)

// A status word carries its flag and count in one 32-bit value and nothing
// else is read on its strength, so relaxed device-scope accesses suffice (no
// fence: publishing does not wait for the tile's earlier scatter writes).
__device__ __forceinline__ uint32_t ld_status(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_status(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int32_t *p) { return *reinterpret_cast<const volatile int32_t *>(p); }

// Adds this thread's digits of key (one digit per pass, pass q at bit
// shift0 + 8 q) to the tile histogram hst[q][256]; a warp whose 32 digits
// agree adds them with one atomic.
template <int NPASS>
__device__ __forceinline__ void tile_digits(uint64_t key, bool ok, int shift0, uint32_t (*hst)[256]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NPASS; q++) {
        const uint32_t d = ok ? (uint32_t)(key >> (shift0 + 8 * q)) & 255u : 0xFFFFFFFFu;
        const uint32_t d0 = __shfl_sync(LFC_FULL, d, 0);
        if (__all_sync(LFC_FULL, d == d0)) {
            if (lane == 0 && d0 != 0xFFFFFFFFu) atomicAdd(&hst[q][d0], 32u);
        } else if (d != 0xFFFFFFFFu) {
            atomicAdd(&hst[q][d], 1u);
        }
    }
}

// Adds a tile histogram to the block's digit totals dhist[b][q][256].
template <int NPASS>
__device__ __forceinline__ void flush_digits(uint32_t (*hst)[256], uint32_t *dhist_b) {
    for (int i = threadIdx.x; i < NPASS * 256; i += blockDim.x) {
        const uint32_t c = (&hst[0][0])[i];
        if (c) atomicAdd(dhist_b + i, c);
    }
}

__global__ void zero_u32_kernel(uint32_t *p, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = 0;
}

// Phase 1 keys: K[v] = bytes v .. v + 7 (cyclic) big-endian, element v.
// Phase 1 sorts the first kPhase1Bytes bytes of every rotation; they sit in
// the top bytes of the 64-bit key, so passes 8 - kPhase1Bytes .. 7 carry them.
constexpr int kPhase1Bytes = LFC_PHASE1_BYTES;

// Also adds the tile's bytes to the block's byte histogram and clears the
// tile's look-back status words in both status arrays (the first pass reads
// array 0 and clears array 1 for the second, and so on). Over all rotations
// of a block, the digit of every pass (one byte of each rotation's prefix)
// takes each byte position of the block exactly once, so the digit totals
// of all 8 passes equal the block's byte histogram: one histogram serves
// every pass.
__global__ void __launch_bounds__(kSortThreads) key8_kernel(const BlockState *__restrict__ st,
                                                            const uint8_t *__restrict__ rle_all,
                                                            uint64_t *__restrict__ K_all, int32_t *__restrict__ V_all,
                                                            uint32_t *__restrict__ dhist_all, uint32_t *__restrict__ lb_all,
                                                            size_t lb_array_words) {
    __shared__ uint8_t sb[kTile + 8];
    __shared__ uint32_t hst[1][256];
    const int b = blockIdx.y, tile = blockIdx.x;
    const int m = st[b].m;
    const int t0 = tile * kTile;
    if (t0 >= m) return;
    const int cnt = min(kTile, m - t0);
    const uint8_t *rle = rle_all + (size_t)b * kBlockCap;
    for (int i = threadIdx.x; i < cnt + 7; i += kSortThreads) sb[i] = rle[(t0 + i) % m];
    hst[0][threadIdx.x] = 0;
    uint32_t *lbt = lb_all + (size_t)b * kLbBlockWords + (size_t)tile * 256;
    lbt[threadIdx.x] = 0;
    lbt[lb_array_words + threadIdx.x] = 0;
    __syncthreads();
    uint64_t *K = K_all + (size_t)b * kBlockCap;
    int32_t *V = V_all + (size_t)b * kBlockCap;
    for (int r = 0; r < kPerThread; r++) {
        const int kl = r * kSortThreads + threadIdx.x;
        const bool ok = kl < cnt;
        uint64_t key = 0;
        if (ok) {
#pragma unroll
            for (int q = 0; q < kPhase1Bytes; q++) key = (key << 8) | sb[kl + q];
            key <<= 8 * (8 - kPhase1Bytes);
            K[t0 + kl] = key;
            V[t0 + kl] = t0 + kl;
        }
        tile_digits<1>((uint64_t)sb[kl], ok, 0, hst);  // the tile's own byte
    }
    __syncthreads();
    flush_digits<1>(hst, dhist_all + (size_t)b * kSweepPasses * 256);
}

// Round words of the tied elements: rank[v] << 40 | rank[(v + h) mod m] << 20 | v.
constexpr uint64_t kElemMask = (1u << 20) - 1u;

__global__ void __launch_bounds__(kSortThreads) key40_kernel(const int32_t *__restrict__ rs, const BlockState *__restrict__ st,
                                                             const int32_t *__restrict__ V_all, const int32_t *__restrict__ rank_all,
                                                             uint64_t *__restrict__ K_all, int32_t *__restrict__ big) {
    if (rs[kRsAbort]) return;
    const int b = blockIdx.y, tile = blockIdx.x;
    const int h = rs[2];
    const BlockState s = st[b];
    const int n = sort_count<1>(s, h);
    if (tile * kTile >= n) return;
    if (tile == 0 && threadIdx.x == 0) big[b] = 0;  // set again by the segmented sort if a group is too large
    const size_t bo = (size_t)b * kBlockCap;
    // all elements first, then all rank gathers (independent loads in flight together)
    int vv[kPerThread];
#pragma unroll
    for (int r = 0; r < kPerThread; r++) {
        const int k = tile * kTile + r * kSortThreads + threadIdx.x;
        vv[r] = k < n ? V_all[bo + k] : -1;
    }
#pragma unroll
    for (int r = 0; r < kPerThread; r++) {
        if (vv[r] < 0) continue;
        const int k = tile * kTile + r * kSortThreads + threadIdx.x, v = vv[r];
        int j = v + h;
        if (j >= s.m) j -= s.m;
        K_all[bo + k] = ((uint64_t)(uint32_t)rank_all[bo + v] << 40) | ((uint64_t)(uint32_t)rank_all[bo + j] << 20) |
                        (uint64_t)(uint32_t)v;
    }
}

// Digit totals of the 5 round passes, for the blocks the segmented sort
// flagged (the only ones that take the radix passes).
__global__ void __launch_bounds__(kSortThreads) round_digits_kernel(const int32_t *__restrict__ rs, const BlockState *__restrict__ st,
                                                                    const uint64_t *__restrict__ K_all, uint32_t *__restrict__ dhist_all,
                                                                    const int32_t *__restrict__ big) {
    __shared__ uint32_t hst[5][256];
    if (rs[kRsAbort]) return;
    const int b = blockIdx.y, tile = blockIdx.x;
    if (!big[b]) return;
    const int n = sort_count<1>(st[b], rs[2]);
    if (tile * kTile >= n) return;
    for (int i = threadIdx.x; i < 5 * 256; i += kSortThreads) (&hst[0][0])[i] = 0;
    __syncthreads();
    const uint64_t *K = K_all + (size_t)b * kBlockCap;
    for (int r = 0; r < kPerThread; r++) {
        const int k = tile * kTile + r * kSortThreads + threadIdx.x;
        const bool ok = k < n;
        tile_digits<5>(ok ? K[k] : 0ull, ok, 20, hst);
    }
    __syncthreads();
    flush_digits<5>(hst, dhist_all + (size_t)b * kSweepPasses * 256);
}

// Work items of the radix passes of a phase or round, tile-major: item i is
// tile i / nblocks of block i % nblocks, so that the tiles in flight spread
// over all blocks and a tile's earlier tiles of the same block have mostly
// finished (a look-back then stops within a few steps). Per block its tile
// count ceil(n_b / kTile) goes to rs[kRsTileOff + b]; rs[kRsItems] = the
// largest count x nblocks (items past a block's last tile are skipped); both
// work queues start empty. One CTA.
// In a round (MODE 1) only the blocks flagged by the segmented sort (a group
// longer than its window) take the radix passes. In phase 1 (MODE 0) it also
// writes row 1 of every block's digit totals: the exclusive prefix of row 0
// (the byte histogram), i.e. the block's elements with a smaller digit, the
// same for every pass and tile.
template <int MODE>
__global__ void __launch_bounds__(1024) sort_items_kernel(int32_t *__restrict__ rs, const BlockState *__restrict__ st, int nblocks,
                                                          const int32_t *__restrict__ big, uint32_t *__restrict__ dhist_all) {
    __shared__ int smax;
    if (MODE == 0) {
        const int lane = threadIdx.x & 31;
        for (int bb = threadIdx.x >> 5; bb < nblocks; bb += blockDim.x >> 5) {
            uint32_t *row = dhist_all + (size_t)bb * kSweepPasses * 256;
            uint32_t c[8], t = 0;
#pragma unroll
            for (int i = 0; i < 8; i++) { c[i] = row[lane * 8 + i]; t += c[i]; }
            uint32_t x = warp_incl_sum(t) - t;
#pragma unroll
            for (int i = 0; i < 8; i++) { row[256 + lane * 8 + i] = x; x += c[i]; }
        }
    }
    const bool abort = rs[kRsAbort] != 0;
    const int h = round_h<MODE>(rs);
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    int mx = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        const bool take = !abort && (MODE == 0 || big[b] != 0);
        const int t = take ? (sort_count<MODE>(st[b], h) + kTile - 1) / kTile : 0;
        rs[kRsTileOff + b] = t;
        mx = max(mx, t);
    }
    atomicMax(&smax, mx);
    __syncthreads();
    if (threadIdx.x == 0) {
        rs[kRsItems] = smax * nblocks;
        rs[kRsQueue] = 0;
        rs[kRsQueue + 1] = 0;
    }
}

// Segmented sort of a doubling round. The tied elements of a block are
// listed in suffix-array order, so their round words rank[v] << 40 |
// rank[v + h] << 20 | v are already sorted by the group rank (the top bits);
// a round only has to order each group by the rest of the word (v breaks the
// ties, which keeps identical rotations in start order). A CTA takes the
// groups whose head lies in its 4096-element tile (the window [lo, hi) runs
// from the first head at or after the tile start to the first head at or
// after the tile end), sorts the window's words in shared memory and writes
// them back to the same indices. Groups of at most kSegSmall elements rank
// each word by counting the smaller words of its group; a window with a larger
// group is sorted whole by a bitonic network. A window longer than kSegCap
// (a group longer than kSegCap - kTile + 1) flags its block, which then takes
// the radix passes instead.
constexpr int kSegCap = 8192;
constexpr int kSegThreads = 512;
constexpr int kSegSmall = 256;
constexpr size_t kSegSmem = (size_t)kSegCap * 8;

// First index in [k, limit) whose group rank differs from r (limit if none);
// read 32 words at a time by one warp (all lanes call it).
__device__ __forceinline__ int next_head(const uint64_t *K, int k, int limit, uint64_t r) {
    const int lane = threadIdx.x & 31;
    for (; k < limit; k += 32) {
        const int i = k + lane;
        const bool diff = i < limit && (K[i] >> 40) != r;
        const uint32_t m = __ballot_sync(LFC_FULL, diff);
        if (m) return k + __ffs(m) - 1;
    }
    return limit;
}

__global__ void __launch_bounds__(kSegThreads) segsort_kernel(const int32_t *__restrict__ rs, const BlockState *__restrict__ st,
                                                              const uint64_t *__restrict__ K_all, uint64_t *__restrict__ Kout_all,
                                                              int32_t *__restrict__ big) {
    extern __shared__ __align__(16) uint64_t sw[];  // [kSegCap]
    __shared__ int s_lo, s_hi, s_gmax;
    __shared__ int s_last[kSegCap / 32], s_first[kSegCap / 32], s_scan[33];
    if (rs[kRsAbort]) return;
    const int b = blockIdx.y, tile = blockIdx.x;
    const int h = rs[2];
    const int n = sort_count<1>(st[b], h);
    const int t0 = tile * kTile;
    if (t0 >= n) return;
    const size_t bo = (size_t)b * kBlockCap;
    const uint64_t *K = K_all + bo;
    if (threadIdx.x < 32) {
        // window: skip the group begun before the tile, extend past the tile end
        // to the end of the last group; every scan stops after kSegCap words
        int lo = t0;
        if (t0 > 0) lo = next_head(K, t0, min(n, t0 + kSegCap), K[t0 - 1] >> 40);
        const int te = min(n, t0 + kTile);
        int hi = te;
        if (lo < te && te < n) hi = next_head(K, te, min(n, lo + kSegCap + 1), K[te - 1] >> 40);
        if (threadIdx.x == 0) {
            s_lo = lo;
            s_hi = hi;
            s_gmax = 0;
        }
    }
    __syncthreads();
    const int lo = s_lo, hi = s_hi, cnt = hi - lo;
    if (cnt <= 0) return;  // the tile lies inside a group begun earlier
    if (cnt > kSegCap || (lo > t0 && lo - t0 >= kSegCap)) {
        if (threadIdx.x == 0) atomicExch(&big[b], 1);
        return;
    }
    for (int i = threadIdx.x; i < cnt; i += kSegThreads) sw[i] = K[lo + i];
    __syncthreads();
    // Group bounds in O(1) per word: word i (thread i % kSegThreads, so a
    // warp holds the 32 consecutive words of a chunk) is a head if its group
    // rank differs from word i - 1's; inside a chunk the last head at or
    // before i and the first head after i come from the warp's ballot of
    // head flags, across chunks from a scan over the chunks' last and first
    // heads (exclusive max going up, exclusive max of cnt - first head going
    // down). Then the word's rank inside its group is the count of the
    // group's smaller words, and the word goes straight to that index of the
    // output (the writes of a window stay inside it). Neighbouring lanes hold
    // neighbouring words of mostly the same group, so the counting reads are
    // broadcasts. A window holding a group longer than kSegSmall is sorted
    // whole below and written again.
    constexpr int kChunks = kSegCap / 32;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kChunks * 32; i += kSegThreads) {
        const bool hd = i < cnt && (i == 0 || (sw[i] >> 40) != (sw[i - 1] >> 40));
        const uint32_t m = __ballot_sync(LFC_FULL, hd);
        if (lane == 0) {
            const int base = i;  // i is the chunk's first word here
            s_last[i >> 5] = m ? base + 31 - __clz(m) : -1;
            s_first[i >> 5] = m ? base + __ffs(m) - 1 : -1;
        }
    }
    __syncthreads();
    {
        const int t = threadIdx.x;
        const int up = t < kChunks ? s_last[t] : -1;
        const int cd = kChunks - 1 - t;  // chunks taken from the top going down
        const int dn = (t < kChunks && s_first[cd] >= 0) ? cnt - s_first[cd] : -1;
        const int before = block_excl_max(up, s_scan);  // last head in a lower chunk
        const int after = block_excl_max(dn, s_scan);   // cnt - first head in a higher chunk
        __syncthreads();
        if (t < kChunks) {
            s_last[t] = before;
            s_first[cd] = after >= 0 ? cnt - after : cnt;
        }
    }
    __syncthreads();
    uint64_t *Kout = Kout_all + bo + lo;
    bool gbig = false;
    const uint32_t le = lanemask_lt() | (1u << lane), gtm = lanemask_gt();
    for (int i0 = (int)(threadIdx.x & ~31u); i0 < cnt; i0 += kSegThreads) {
        const int i = i0 + lane;
        const bool in = i < cnt;
        const uint64_t w = in ? sw[i] : 0ull;
        const bool hd = in && (i == 0 || (w >> 40) != (sw[i - 1] >> 40));
        const uint32_t m = __ballot_sync(LFC_FULL, hd);
        if (!in) continue;
        const uint32_t ml = m & le, mg = m & gtm;
        const int gs = ml ? i0 + 31 - __clz(ml) : s_last[i0 >> 5];
        const int ge = mg ? i0 + __ffs(mg) - 1 : s_first[i0 >> 5];
        if (ge - gs > kSegSmall) {
            gbig = true;
        } else {
            int c = gs;
            for (int j = gs; j < ge; j++) c += sw[j] < w;
            Kout[c] = w;
        }
    }
    if (gbig) s_gmax = kSegSmall + 1;
    __syncthreads();
    if (s_gmax > kSegSmall) {
        // bitonic sort of the whole window, padded to a power of two
        int np = 1;
        while (np < cnt) np <<= 1;
        for (int i = cnt + threadIdx.x; i < np; i += kSegThreads) sw[i] = ~0ull;
        __syncthreads();
        for (int k = 2; k <= np; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < np; i += kSegThreads) {
                    const int l = i ^ j;
                    if (l > i) {
                        const uint64_t x = sw[i], y = sw[l];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) {
                            sw[i] = y;
                            sw[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < cnt; i += kSegThreads) Kout[i] = sw[i];
    }
}

// Digit position of a pass: phase 1 sorts all 64 key bits, a round bits 20..59.
template <int MODE>
__device__ __forceinline__ int digit_shift(int pass) { return (MODE == 0 ? 0 : 20) + 8 * pass; }

// One stable LSD pass of (key, element) pairs (MODE 0) or round words (MODE
// 1, the element rides in the word) over every block of the pass.
// Persistent: CTAs take tiles from the pass's work queue until it is empty
// (tile-major order, see sort_items_kernel).
// Per tile: warp w ranks elements [w*512, (w+1)*512) of the tile 32 at a
// time in order (equal digits by __match_any_sync and a per-warp running
// count), giving the tile's count c[d] of every digit d; thread d publishes
// c[d] (flag "aggregate"; tile 0: "inclusive"), adds the published counts of
// the block's earlier tiles back to the nearest "inclusive" one, publishes
// its own inclusive count, and the run of digit d starts at (elements of the
// block with a smaller digit: in phase 1 the offsets sort_items_kernel
// derived from the block's byte histogram, in a round a scan of the pass's
// digit totals) + (elements of digit d in earlier tiles). A CTA takes its
// next work item while it sorts the current one. Tiles are placed in shared memory in digit
// order and each digit's run is written with consecutive threads on
// consecutive addresses.
// A tile waits only on tiles taken from the queue before it, which are held
// by running CTAs, so the waits always end; each is still bounded by
// `budget` clock cycles, after which the CTA raises the abort word and every
// sort kernel of this suffix sort returns at once (LFC_ERR_TIMEOUT).
// Status words of the pass live in array par = pass parity; each tile clears
// its words in the other array for the next pass (which runs on the same or
// fewer tiles of every block).
constexpr size_t kScatterSmem = (size_t)kTile * 12 + (size_t)(kSortThreads / 32) * 256 * 4 + 2 * 256 * 4;
// MODE 1 moves the words alone (Vin / Vout unused)
constexpr size_t kScatterSmem1 = (size_t)kTile * 8 + (size_t)(kSortThreads / 32) * 256 * 4 + 2 * 256 * 4;
constexpr int kSweepCtasPerSm = 3;

template <int MODE>
__global__ void __launch_bounds__(kSortThreads, kSweepCtasPerSm)
radix_sweep_kernel(int pass, int nblocks, int32_t *__restrict__ rs, const BlockState *__restrict__ st,
                   const uint64_t *__restrict__ Kin_all, const int32_t *__restrict__ Vin_all,
                   uint64_t *__restrict__ Kout_all, int32_t *__restrict__ Vout_all,
                   const uint32_t *__restrict__ dhist_all, uint32_t *__restrict__ lb_all, size_t lb_array_words,
                   long long budget) {
    constexpr int NW = kSortThreads / 32;
    extern __shared__ __align__(16) uint8_t smem[];
    uint64_t *sK = reinterpret_cast<uint64_t *>(smem);           // [kTile]
    int32_t *sV = reinterpret_cast<int32_t *>(sK + kTile);        // [kTile], MODE 0
    uint32_t *wcnt = reinterpret_cast<uint32_t *>(MODE == 0 ? reinterpret_cast<uint8_t *>(sV + kTile)
                                                            : reinterpret_cast<uint8_t *>(sK + kTile));  // [NW][256]
    uint32_t *loff = wcnt + NW * 256;                             // [256] tile-local start of a digit
    uint32_t *gbase = loff + 256;                                 // [256] global start of the tile's run
    __shared__ uint32_t sh[33];
    __shared__ int s_item, s_abort, s_fault;
    const int h = round_h<MODE>(rs);
    const int par = MODE == 0 ? (pass & 1) : ((rs[kRsRound] + pass) & 1);
    uint32_t *lb = lb_all + (size_t)par * lb_array_words;
    uint32_t *lb_next = lb_all + (size_t)(par ^ 1) * lb_array_words;
    int32_t *queue = rs + kRsQueue + par;
    if (blockIdx.x == 0 && threadIdx.x == 0) rs[kRsQueue + (par ^ 1)] = 0;  // the next pass's queue
    const int total = rs[kRsItems];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, d = threadIdx.x;
    const int shift = digit_shift<MODE>(pass);
    const uint32_t lt = lanemask_lt(), gt = lanemask_gt();
    // the next work item is taken while the current one is sorted (its ticket
    // is larger, so every tile still only waits on tiles taken before it)
    int nxt = 0;
    if (threadIdx.x == 0) nxt = atomicAdd(queue, 1);
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = nxt;
            s_abort = ld_volatile_i32(rs + kRsAbort);
            s_fault = ld_volatile_i32(rs + kRsFault);
            nxt = atomicAdd(queue, 1);
        }
        for (int i = threadIdx.x; i < NW * 256; i += kSortThreads) wcnt[i] = 0;
        __syncthreads();
        const int item = s_item;
        if (item >= total || s_abort) break;
        const int tile = item / nblocks, b = item - tile * nblocks;
        if (tile >= rs[kRsTileOff + b]) {  // past the block's last tile
            __syncthreads();
            continue;
        }
        const int n = sort_count<MODE>(st[b], h);
        const size_t bo = (size_t)b * kBlockCap;
        // phase 1: the block's elements with a smaller digit (row 1, see sort_items_kernel)
        const uint32_t below1 = MODE == 0 ? dhist_all[((size_t)b * kSweepPasses + 1) * 256 + d] : 0u;
        const uint64_t *Kin = Kin_all + bo;
        const int32_t *Vin = Vin_all + bo;
        uint64_t keys[kPerThread];
        int32_t vals[kPerThread];
        uint32_t rnk[kPerThread];
#pragma unroll
        for (int r = 0; r < kPerThread; r++) {
            const int k = tile * kTile + w * 512 + r * 32 + lane;
            const bool ok = k < n;
            keys[r] = ok ? Kin[k] : 0;
            vals[r] = (MODE == 0 && ok) ? Vin[k] : 0;
            const uint32_t dg = (uint32_t)(keys[r] >> shift) & 255u;
            const uint32_t mm = __match_any_sync(LFC_FULL, ok ? dg : 256u + lane);
            uint32_t before = 0;
            if (ok) before = wcnt[w * 256 + dg];
            __syncwarp();
            if (ok && (mm & gt) == 0) wcnt[w * 256 + dg] = before + __popc(mm);
            __syncwarp();
            rnk[r] = ok ? before + __popc(mm & lt) : 0xFFFFFFFFu;
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, the tile's count, then over digits
        uint32_t cnt_d = 0;
        for (int ww = 0; ww < NW; ww++) {
            const uint32_t c = wcnt[ww * 256 + d];
            wcnt[ww * 256 + d] = cnt_d;
            cnt_d += c;
        }
        loff[d] = block_excl_sum<uint32_t>(cnt_d, sh, nullptr);
        // decoupled look-back over the block's earlier tiles
        uint32_t *lbb = lb + (size_t)b * kLbBlockWords;
        const bool withhold = s_fault != 0 && b == 0 && tile == 0;  // fault injection: never publish
        if (!withhold) st_status(lbb + (size_t)tile * 256 + d, (tile == 0 ? kLbIncl : kLbAgg) | cnt_d);
        uint32_t excl = 0;
        bool gave_up = false;
        if (tile > 0) {
            const long long t0 = clock64();
            int tp = tile - 1;
            for (;;) {
                const uint32_t sv = ld_status(lbb + (size_t)tp * 256 + d);
                if (sv & (kLbAgg | kLbIncl)) {
                    excl += sv & kLbCount;
                    if ((sv & kLbIncl) || tp == 0) break;
                    tp--;
                    continue;
                }
                if (ld_volatile_i32(rs + kRsAbort)) { gave_up = true; break; }
                if (clock64() - t0 > budget) {
                    gave_up = true;
                    atomicCAS(rs + kRsAbort, 0, (int)LFC_ERR_TIMEOUT);
                    atomicCAS(rs + kRsSticky, 0, (int)LFC_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
            if (!gave_up) st_status(lbb + (size_t)tile * 256 + d, kLbIncl | (excl + cnt_d));
        }
        lb_next[(size_t)b * kLbBlockWords + (size_t)tile * 256 + d] = 0;
        const uint32_t below = MODE == 0 ? below1
                                         : block_excl_sum<uint32_t>(dhist_all[((size_t)b * kSweepPasses + pass) * 256 + d],
                                                                    sh, nullptr);  // block elements with a smaller digit
        gbase[d] = below + excl;
        if (withhold && d == 0) atomicExch(rs + kRsFault, 0);  // the fault fires once
        if (__syncthreads_or(gave_up)) break;
#pragma unroll
        for (int r = 0; r < kPerThread; r++) {
            if (rnk[r] == 0xFFFFFFFFu) continue;
            const uint32_t dg = (uint32_t)(keys[r] >> shift) & 255u;
            const uint32_t pos = loff[dg] + wcnt[w * 256 + dg] + rnk[r];
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
                const uint32_t dg = (uint32_t)(key >> shift) & 255u;
                const uint32_t g = gbase[dg] + ((uint32_t)j - loff[dg]);
                Kout[g] = key;
                if (MODE == 0) Vout[g] = sV[j];
            }
        }
        __syncthreads();
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
    if (rs[kRsAbort]) return;
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
    if (rs[kRsAbort]) return;
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
// next round's lists. A thread walks 16 consecutive elements for the scans
// (the last head before each element, the compacted offsets) and stages per
// element its group's head and its offset in the compacted lists (-1: not
// tied) in shared memory; the outputs are then written by consecutive
// threads on consecutive elements, so the suffix-array and list stores are
// coalesced (only rank[v] is a scatter).
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }  // conflict-free for both access patterns

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
    __shared__ int32_t s_head[kTile + kTile / 32];  // head position of the element's group
    __shared__ int32_t s_off[kTile + kTile / 32];   // offset in the compacted lists, -1: not tied
    if (rs[kRsAbort]) return;
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
    const int t0 = tile * kTile;
    const int kl0 = threadIdx.x * kPerThread;
    const int k0 = t0 + kl0;
    const int k1 = min(n, k0 + kPerThread);
    int mine = -1, tied = 0;
    // a full run loads flags and positions with 16-byte loads; the block
    // scans are reached by every thread
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
#pragma unroll
        for (int q = 0; q < kPerThread; q++) {
            const bool hd = (fw[q >> 2] >> (8 * (q & 3))) & 1u;
            const bool nh = q + 1 < kPerThread ? ((fw[(q + 1) >> 2] >> (8 * ((q + 1) & 3))) & 1u) : last_next;
            if (hd) carry = pv[q];
            s_head[pad32(kl0 + q)] = carry;
            s_off[pad32(kl0 + q)] = (hd && nh) ? -1 : off++;
        }
    } else {
        for (int k = k0; k < k1; k++) {
            const bool hd = flags[k];
            const bool nh = (k + 1 >= n) || flags[k + 1];
            if (hd) carry = MODE == 0 ? k : act[k];
            s_head[pad32(k - t0)] = carry;
            s_off[pad32(k - t0)] = (hd && nh) ? -1 : off++;
        }
    }
    __syncthreads();
    const int cnt = min(kTile, n - t0);
    for (int j = threadIdx.x; j < cnt; j += kSortThreads) {
        const int k = t0 + j;
        const int pos = MODE == 0 ? k : act[k];
        const int32_t v = MODE == 0 ? sorted[k] : (int32_t)(words[k] & kElemMask);
        rank[v] = s_head[pad32(j)];
        if (MODE == 1 || sorted != sa) sa[pos] = v;
        const int o = s_off[pad32(j)];
        if (o >= 0) {
            act_out[o] = pos;
            val_out[o] = v;
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
// while tied elements remain, h is below the largest block length and no
// wait has given up.
__global__ void round_end_kernel(int32_t *rs, int max_m, cudaGraphConditionalHandle cond, int set_cond) {
    rs[2] *= 2;
    rs[3] += 1;
    if (set_cond) cudaGraphSetConditional(cond, (rs[kRsAbort] == 0 && rs[0] > 0 && rs[2] < max_m) ? 1u : 0u);
}

// L[j] = block[(SA[j] - 1) mod m]; origPtr = j with SA[j] = 0; bytes in use.
// Each CTA also writes the MTF summary of its 4096-byte segment of L: the
// distinct bytes ordered by last occurrence, latest first. Thread = 16
// consecutive positions; the last position of each byte value comes from one
// shared-memory max per distinct value of a thread's run; each value is then
// marked at its last position and the marks are compacted from the top.
// After an aborted sort the suffix array is incomplete: the kernel then
// takes the identity order instead, so that every later stage still reads
// in-range values (the call reports LFC_ERR_TIMEOUT and its output is void).
__global__ void __launch_bounds__(kSortThreads) bwt_output_kernel(BlockState *__restrict__ st, const int32_t *__restrict__ sa_all,
                                                                  const uint8_t *__restrict__ rle_all, uint8_t *__restrict__ L_all,
                                                                  uint8_t *__restrict__ rec_all, int32_t *__restrict__ reclen_all,
                                                                  const int32_t *__restrict__ rs) {
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
    if (rs[kRsAbort]) {
#pragma unroll
        for (int q = 0; q < kPerThread; q++) sv[q] = j0 + q < m ? j0 + q : -1;
    } else if (j0 + kPerThread <= m) {  // full run: the suffix array by 16-byte loads
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

// Copies every block's last column out (lfc_bwt_blocks): stride bytes per
// block, its length (the RLE1 length) and its origin row.
__global__ void copy_bwt_kernel(const BlockState *__restrict__ st, const uint8_t *__restrict__ L_all, uint8_t *__restrict__ out,
                                size_t stride, uint32_t *__restrict__ len, uint32_t *__restrict__ orig) {
    const int b = blockIdx.y;
    const int m = st[b].m;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        len[b] = (uint32_t)m;
        orig[b] = (uint32_t)st[b].orig_ptr;
    }
    const uint8_t *src = L_all + (size_t)b * kBlockCap;
    uint8_t *dst = out + (size_t)b * stride;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

cudaError_t launch_copy_bwt(lfc_plan P, int nblocks, uint8_t *d_L, size_t stride, uint32_t *d_len, uint32_t *d_orig) {
    copy_bwt_kernel<<<dim3(64, nblocks), 256, 0, P->stream>>>(P->ws.bstate, P->ws.bwt, d_L, stride, d_len, d_orig);
    count_launches(P, 1);
    return cudaGetLastError();
}

template <int MODE>
static void sweep_pass(lfc_plan P, cudaStream_t st, int nblocks, int ctas, int pass, const uint64_t *kin, const int32_t *vin,
                       uint64_t *kout, int32_t *vout) {
    Workspace &ws = P->ws;
    radix_sweep_kernel<MODE><<<ctas, kSortThreads, MODE == 0 ? kScatterSmem : kScatterSmem1, st>>>(
        pass, nblocks, ws.act_total, ws.bstate, kin, vin, kout, vout, ws.dhist, ws.lbstat, ws.lbstat_words,
        P->wait_cycles);
    count_launches(P, 1);
}

static int sweep_ctas(lfc_plan P, int nblocks, int tiles) {
    const long long items = (long long)nblocks * tiles;
    const long long cap = (long long)P->sm_count * kSweepCtasPerSm;
    return (int)std::max<long long>(1, std::min(items, cap));
}

// One prefix-doubling round over the tied elements (h and the parity of the
// active lists come from the round state in device memory).
static void bwt_round(lfc_plan P, cudaStream_t st, int nblocks, int tiles, int max_m, cudaGraphConditionalHandle cond,
                      int set_cond) {
    Workspace &ws = P->ws;
    round_start_kernel<<<1, 1, 0, st>>>(ws.act_total, 0);
    const size_t nd = (size_t)nblocks * kSweepPasses * 256;
    zero_u32_kernel<<<(unsigned)std::min<size_t>(64, (nd + 255) / 256), 256, 0, st>>>(ws.dhist, nd);
    dim3 g1(tiles, nblocks);
    key40_kernel<<<g1, kSortThreads, 0, st>>>(ws.act_total, ws.bstate, ws.val, ws.rank, ws.keys, ws.segbig);
    // groups within their windows: keys -> keys2 directly; blocks with a
    // longer group are flagged and take the 5 LSD passes over bits 20..59 of
    // the words instead: keys -> keys2 -> ... -> keys2
    segsort_kernel<<<g1, kSegThreads, kSegSmem, st>>>(ws.act_total, ws.bstate, ws.keys, ws.keys2, ws.segbig);
    round_digits_kernel<<<g1, kSortThreads, 0, st>>>(ws.act_total, ws.bstate, ws.keys, ws.dhist, ws.segbig);
    sort_items_kernel<1><<<1, 1024, 0, st>>>(ws.act_total, ws.bstate, nblocks, ws.segbig, nullptr);
    count_launches(P, 6);
    const int ctas = sweep_ctas(P, nblocks, tiles);
    for (int pass = 0; pass < 5; pass++) {
        if (pass & 1) sweep_pass<1>(P, st, nblocks, ctas, pass, ws.keys2, nullptr, ws.keys, nullptr);
        else sweep_pass<1>(P, st, nblocks, ctas, pass, ws.keys, nullptr, ws.keys2, nullptr);
    }
    heads_tile_kernel<1><<<g1, kSortThreads, 0, st>>>(ws.act_total, ws.bstate, ws.keys2, ws.act, ws.act2, ws.bwt,
                                                      ws.tileaux);
    heads_scan_kernel<1><<<nblocks, 256, 0, st>>>(ws.act_total, ws.bstate, ws.tileaux);
    heads_apply_kernel<1><<<g1, kSortThreads, 0, st>>>(ws.act_total, ws.bstate, nullptr, ws.keys2, ws.act, ws.act2,
                                                       ws.bwt, ws.tileaux, ws.rank, ws.sa, ws.val);
    commit_round_kernel<<<(nblocks + 255) / 256, 256, 0, st>>>(ws.bstate, nblocks);
    round_end_kernel<<<1, 1, 0, st>>>(ws.act_total, max_m, cond, set_cond);
    count_launches(P, 5);
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
    e = cudaFuncSetAttribute(radix_sweep_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(radix_sweep_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(segsort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSegSmem);
    if (e != cudaSuccess) return e;
    // a new suffix sort: no wait has given up yet (outside graphs the sticky
    // status is reported by this call, so it starts clear as well)
    e = cudaMemsetAsync(ws.act_total + kRsAbort, 0, sizeof(int32_t), s);
    if (e == cudaSuccess && !graph) e = cudaMemsetAsync(ws.act_total + kRsSticky, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    // phase 1: prefix keys and the digit totals of all passes, then 8 LSD
    // passes (keys, sa) -> (keys2, sa2) -> ... -> (keys, sa)
    stage_begin(P, LFC_STAGE_BWT_KEYS);
    dim3 grid(tiles, nblocks);
    const size_t nd = (size_t)nblocks * kSweepPasses * 256;
    zero_u32_kernel<<<(unsigned)std::min<size_t>(64, (nd + 255) / 256), 256, 0, s>>>(ws.dhist, nd);
    key8_kernel<<<grid, kSortThreads, 0, s>>>(ws.bstate, ws.rle, ws.keys, ws.sa, ws.dhist, ws.lbstat, ws.lbstat_words);
    sort_items_kernel<0><<<1, 1024, 0, s>>>(ws.act_total, ws.bstate, nblocks, nullptr, ws.dhist);
    count_launches(P, 3);
    uint64_t *kin = ws.keys, *kout = ws.keys2;
    int32_t *vin = ws.sa, *vout = ws.sa2;
    stage_end(P, LFC_STAGE_BWT_KEYS);
    stage_begin(P, LFC_STAGE_BWT_SORT8);
    const int ctas = sweep_ctas(P, nblocks, tiles);
    for (int pass = 8 - kPhase1Bytes; pass < 8; pass++) {
        sweep_pass<0>(P, s, nblocks, ctas, pass, kin, vin, kout, vout);
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
        e = cudaMemcpyAsync(ws.h_act_total, ws.act_total, kSortCtlHead * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        int round = 0;
        for (int h = kPhase1Bytes; ws.h_act_total[kRsAbort] == 0 && ws.h_act_total[0] > 0 && h < max_m; h *= 2, round++) {
            P->bwt_rounds++;
            P->bwt_tied_total += ws.h_act_total[0];
            if (round < 32) P->bwt_round_tied[round] += ws.h_act_total[0];
            const int t1 = (ws.h_act_total[1] + kTile - 1) / kTile;
            bwt_round(P, s, nblocks, t1, max_m, cudaGraphConditionalHandle{}, 0);
            e = cudaMemcpyAsync(ws.h_act_total, ws.act_total, kSortCtlHead * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return e;
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
        }
        if (ws.h_act_total[kRsAbort] != 0) P->bwt_timed_out = true;
    }
    stage_end(P, LFC_STAGE_BWT_REFINE);
    stage_begin(P, LFC_STAGE_BWT_OUT);
    bwt_output_kernel<<<grid, kSortThreads, 0, s>>>(ws.bstate, ws.sa, ws.rle, ws.bwt, ws.mtfrec, ws.mtfreclen,
                                                     ws.act_total);
    stage_end(P, LFC_STAGE_BWT_OUT);
    count_launches(P, 1);
    return cudaGetLastError();
}

}  // namespace lfc

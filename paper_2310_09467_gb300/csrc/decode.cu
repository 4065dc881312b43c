// decode.cu -- decompression (Fig. 2b: unpack the header, bzip2-decode every
// block, then the inverse predictor chosen by the header's id).
//
// One CTA per bzip2 stream. Every read of the coded stream is checked
// against its length and every write against its buffer, so corrupt input
// ends in an error flag, never an out-of-bounds access.
//  1. thread 0: headers and tables; the CTA: Huffman lookup tables (a
//     symbol per 10-bit prefix; whole-code counts and lengths per 12-bit
//     prefix); thread 0 walks the groups of 50 codes for their bit offsets
//     (EOB lies in the last group, as an encoder writes one selector per
//     group it uses: a stream with more selectors is rejected as corrupt);
//     every thread decodes whole groups into the symbol array; inverse
//     RUNA/RUNB and MTF by 32 segments (each segment's moves permute list
//     positions whatever the list holds: permutations first, then the lists
//     at the segment starts in order, then every segment decoded) -> the BWT
//     last column L;
//  2. the CTA: LF mapping T[j] = C[L[j]] + rank of j among equal bytes (a
//     stable counting sort of L with per-warp counters);
//  3. 1024 walkers invert the BWT: each starts at its own row (walker 0 at
//     origPtr), follows T until it meets another walker's start row, the
//     pieces are chained from walker 0, and every walker re-walks its piece
//     writing bytes from the end of the block backwards;
//  4. the CTA: inverse RLE1 from sync points (one piece per thread), then
//     CRC-32/BZIP2 of the output vs the stored block CRC.
#include <climits>

#include "lfc_common.cuh"

namespace lfc {

constexpr int kDecThreads = 1024;
constexpr int kWalkers = kDecThreads;
constexpr uint32_t kPolyD = 0x04C11DB7u;

enum : int32_t {
    DEC_OK = 0, DEC_BAD_MAGIC = 1, DEC_TRUNC = 2, DEC_BAD_TABLE = 3, DEC_BAD_DATA = 4,
    DEC_OVERFLOW = 5, DEC_BAD_ORIG = 6, DEC_BAD_LEN = 7, DEC_BAD_CRC = 8, DEC_BAD_WALK = 9
};

constexpr int kDecWarps = kDecThreads / 32;       // MTF segments per block

struct DecBlock {
    const uint8_t *src;   // one standalone bzip2 stream
    int64_t src_len;
    uint8_t *dst;         // decoded bytes go here
    int32_t expect;       // decoded length the container promises
    int32_t pad;
};

// MSB-first bit reader over a bounded byte string: up to 64 bits buffered
// left-aligned, each byte loaded once. get(k) (k <= 32) past the end sets
// err and returns 0; peek(k) pads with zeros past the end.
struct BitReader {
    const uint8_t *p;
    int64_t nbytes, next;  // bytes in the string, next byte to load
    uint64_t buf;          // buffered bits, left-aligned
    int bcnt;              // buffered bit count
    bool err;
    __device__ void init(const uint8_t *src, int64_t n) {
        p = src;
        nbytes = n;
        next = 0;
        buf = 0;
        bcnt = 0;
        err = false;
    }
    // Called with fewer bits buffered than a read needs (at most 32): 32
    // more bits from four independent loads (one memory latency, not four);
    // the last bytes of the string one by one
    __device__ __forceinline__ void refill() {
        if (bcnt <= 32 && next + 4 <= nbytes) {
            const uint32_t w = ((uint32_t)__ldg(p + next) << 24) | ((uint32_t)__ldg(p + next + 1) << 16) |
                               ((uint32_t)__ldg(p + next + 2) << 8) | (uint32_t)__ldg(p + next + 3);
            buf |= (uint64_t)w << (32 - bcnt);
            bcnt += 32;
            next += 4;
            return;
        }
        while (bcnt <= 56 && next < nbytes) {
            buf |= (uint64_t)__ldg(p + next++) << (56 - bcnt);
            bcnt += 8;
        }
    }
    __device__ __forceinline__ uint32_t peek(int k) {
        if (bcnt < k) refill();
        return (uint32_t)(buf >> (64 - k));
    }
    __device__ __forceinline__ bool skip(int k) {
        if (bcnt < k) refill();
        if (bcnt < k) { err = true; bcnt = 0; buf = 0; return false; }
        buf <<= k;
        bcnt -= k;
        return true;
    }
    __device__ __forceinline__ uint32_t get(int k) {
        const uint32_t v = peek(k);
        return skip(k) ? v : 0u;
    }
};

__device__ __forceinline__ uint32_t gf_mul(uint32_t a, uint32_t b) {
    uint32_t r = 0;
    for (int i = 31; i >= 0; i--) {
        r = (r & 0x80000000u) ? (r << 1) ^ kPolyD : (r << 1);
        if ((b >> i) & 1u) r ^= a;
    }
    return r;
}
__device__ __forceinline__ uint32_t xpow8(uint64_t k) {
    uint32_t r = 1u, b = 0x100u;
    while (k) {
        if (k & 1) r = gf_mul(r, b);
        b = gf_mul(b, b);
        k >>= 1;
    }
    return r;
}

struct DecShared {
    uint32_t crc_tab[256];
    uint32_t warp_cnt[kDecThreads / 32][256];
    uint32_t C[256];
    int32_t walk_next[kWalkers];
    int32_t walk_len[kWalkers];
    int64_t walk_pos[kWalkers];
    uint8_t seq_to_unseq[256];
    uint8_t mtf[256];
    uint8_t sel_list[8];
    uint8_t len[6][258];
    int32_t first[6][22], count[6][22], pidx[6][22];
    uint16_t perm[6][258];
    uint16_t lut[6][1 << 10];  // next 10 bits -> (symbol << 5) | code length, 0: longer code
    uint16_t mlut[6][1 << 12]; // next 12 bits -> (codes << 5) | their bits: the whole codes (at most 4) in them, 0: the first is longer
    BitReader br;              // the header reader, handed from the parse to the decode loop
    int32_t alpha, block_max;
    uint32_t red[32];
    int32_t status, nblock, orig, n_in_use, n_groups, n_sel, out_len;
    uint32_t stored_crc;
    int32_t nsym, ngroups_used;            // Huffman symbols up to EOB, groups holding them
    int32_t seg_start[kDecWarps];          // MTF segment of warp w: [seg_start[w], next start)
    int32_t seg_len[kDecWarps], seg_off[kDecWarps];  // its output bytes and their offset in L
    int32_t seg_status[kDecWarps];
    uint8_t seg_perm[kDecWarps][256];      // where the segment's MTF moves take each list position
    uint8_t seg_list[kDecWarps][256];      // the list at the segment's start
    int32_t scan_sh[33];        // block scan scratch
};

// BitReader whose next 4 bytes are loaded one refill ahead, so a refill
// does not wait for memory (for the one thread that walks all groups).
struct AheadReader : BitReader {
    uint32_t pf;  // bytes next .. next + 3, big-endian (when next + 4 <= nbytes)
    __device__ __forceinline__ uint32_t load4(int64_t at) const {
        return ((uint32_t)__ldg(p + at) << 24) | ((uint32_t)__ldg(p + at + 1) << 16) |
               ((uint32_t)__ldg(p + at + 2) << 8) | (uint32_t)__ldg(p + at + 3);
    }
    __device__ void start(const BitReader &r) {
        *static_cast<BitReader *>(this) = r;
        pf = next + 4 <= nbytes ? load4(next) : 0u;
    }
    __device__ __forceinline__ void refill() {
        if (bcnt <= 32 && next + 4 <= nbytes) {
            buf |= (uint64_t)pf << (32 - bcnt);
            bcnt += 32;
            next += 4;
            pf = next + 4 <= nbytes ? load4(next) : 0u;  // used at the next refill
            return;
        }
        while (bcnt <= 56 && next < nbytes) {
            buf |= (uint64_t)__ldg(p + next++) << (56 - bcnt);
            bcnt += 8;
        }
    }
    __device__ __forceinline__ uint32_t peek(int k) {
        if (bcnt < k) refill();
        return (uint32_t)(buf >> (64 - k));
    }
    __device__ __forceinline__ bool skip(int k) {
        if (bcnt < k) refill();
        if (bcnt < k) { err = true; bcnt = 0; buf = 0; return false; }
        buf <<= k;
        bcnt -= k;
        return true;
    }
    __device__ __forceinline__ uint32_t get(int k) {
        const uint32_t v = peek(k);
        return skip(k) ? v : 0u;
    }
};

// One Huffman symbol with table t: the 10-bit lookup, else the canonical
// search from 11 bits; -1 for a code that is not in the table or a stream
// that ends first (br.err).
template <class Reader>
__device__ __forceinline__ int huff_symbol(Reader &br, const DecShared &S, int t) {
    const uint32_t e = S.lut[t][br.peek(10)];
    if (e) return br.skip(e & 31) ? (int)(e >> 5) : -1;
    int32_t c = (int32_t)br.peek(10);
    if (!br.skip(10)) return -1;
    for (int l = 11; l <= 20; l++) {
        c = (c << 1) | (int32_t)br.get(1);
        if (br.err) return -1;
        const uint32_t d = (uint32_t)(c - S.first[t][l]);
        if (d < (uint32_t)S.count[t][l]) return S.perm[t][S.pidx[t][l] + (int)d];
    }
    return -1;
}

// Workspace per block: sel (kMaxSelectors bytes), L (kBlockCap), T (int32
// kBlockCap), rowmark (int32 kBlockCap, walker id or -1), blk (kBlockCap).
// 64 registers at most, so that a CTA of kDecThreads = 1024 fits an SM.
__global__ void __maxnreg__(64) bzip2_decode_kernel(const DecBlock *__restrict__ blocks, int32_t *__restrict__ status,
                                                                   uint8_t *__restrict__ sel_all, uint8_t *__restrict__ L_all,
                                                                   int32_t *__restrict__ T_all, int32_t *__restrict__ mark_all,
                                                                   uint8_t *__restrict__ blk_all) {
    extern __shared__ __align__(16) uint8_t smraw[];
    DecShared &S = *reinterpret_cast<DecShared *>(smraw);
    const int b = blockIdx.x;
    const DecBlock D = blocks[b];
    uint8_t *sel = sel_all + (size_t)b * kMaxSelectors;
    uint8_t *L = L_all + (size_t)b * kBlockCap;
    int32_t *T = T_all + (size_t)b * kBlockCap;
    int32_t *mark = mark_all + (size_t)b * kBlockCap;
    uint8_t *blk = blk_all + (size_t)b * kBlockCap;
    const int tid = threadIdx.x;
    for (int i = tid; i < 256; i += blockDim.x) {
        uint32_t v = (uint32_t)i << 24;
        for (int k = 0; k < 8; k++) v = (v & 0x80000000u) ? (v << 1) ^ kPolyD : (v << 1);
        S.crc_tab[i] = v;
    }
    if (tid == 0) {
        S.status = DEC_OK;
        BitReader br;
        br.init(D.src, D.src_len);
        int st = DEC_OK;
        do {
            if (br.get(8) != 'B' || br.get(8) != 'Z' || br.get(8) != 'h') { st = DEC_BAD_MAGIC; break; }
            const uint32_t lvl = br.get(8);
            if (lvl < '1' || lvl > '9') { st = DEC_BAD_MAGIC; break; }
            const int block_max = 100000 * (int)(lvl - '0');
            if (br.get(24) != 0x314159u || br.get(24) != 0x265359u) { st = DEC_BAD_MAGIC; break; }
            S.stored_crc = br.get(32);
            if (br.get(1) != 0) { st = DEC_BAD_DATA; break; }
            const int orig = (int)br.get(24);
            const uint32_t used16 = br.get(16);
            int niu = 0;
            for (int i = 0; i < 16; i++) {
                if (!(used16 & (1u << (15 - i)))) continue;
                const uint32_t bits = br.get(16);
                for (int j = 0; j < 16; j++)
                    if (bits & (1u << (15 - j))) S.seq_to_unseq[niu++] = (uint8_t)(i * 16 + j);
            }
            if (br.err) { st = DEC_TRUNC; break; }
            if (niu == 0) { st = DEC_BAD_TABLE; break; }
            const int alpha = niu + 2;
            const int ng = (int)br.get(3);
            const int nsel = (int)br.get(15);
            if (br.err) { st = DEC_TRUNC; break; }
            if (ng < 2 || ng > 6 || nsel < 1 || nsel > kMaxSelectors) { st = DEC_BAD_TABLE; break; }
            for (int t = 0; t < ng; t++) S.sel_list[t] = (uint8_t)t;
            for (int i = 0; i < nsel && st == DEC_OK; i++) {
                int j = 0;
                while (br.get(1)) {
                    if (++j >= ng) { st = DEC_BAD_TABLE; break; }
                }
                if (br.err) st = DEC_TRUNC;
                if (st != DEC_OK) break;
                const uint8_t v = S.sel_list[j];
                for (int q = j; q > 0; q--) S.sel_list[q] = S.sel_list[q - 1];
                S.sel_list[0] = v;
                sel[i] = v;
            }
            if (st != DEC_OK) break;
            for (int t = 0; t < ng && st == DEC_OK; t++) {
                int cur = (int)br.get(5);
                for (int v = 0; v < alpha && st == DEC_OK; v++) {
                    for (;;) {
                        if (cur < 1 || cur > 20 || br.err) { st = br.err ? DEC_TRUNC : DEC_BAD_TABLE; break; }
                        if (!br.get(1)) break;
                        cur += br.get(1) ? -1 : 1;
                    }
                    S.len[t][v] = (uint8_t)cur;
                }
            }
            if (st != DEC_OK) break;
            // canonical tables: the codes of length l are first[l] ..
            // first[l] + count[l] - 1, in increasing symbol order
            for (int t = 0; t < ng; t++) {
                int np = 0;
                int32_t code = 0;
                for (int l = 1; l <= 20; l++) {
                    S.first[t][l] = code;
                    S.pidx[t][l] = np;
                    int cnt = 0;
                    for (int v = 0; v < alpha; v++)
                        if (S.len[t][v] == l) { S.perm[t][np++] = (uint16_t)v; cnt++; }
                    S.count[t][l] = cnt;
                    code = (code + cnt) << 1;
                }
            }
            S.n_in_use = niu;
            S.n_groups = ng;
            S.n_sel = nsel;
            S.alpha = alpha;
            S.block_max = block_max;
            S.orig = orig;
            S.br = br;
        } while (0);
        S.status = st;
    }
    __syncthreads();
    if (S.status != DEC_OK) {
        if (tid == 0) status[b] = S.status;
        return;
    }
    // lookup tables: entry i of table t decodes the code whose first bits are
    // i (as 10 bits), if that code is at most 10 bits long
    for (int q = tid; q < S.n_groups * 1024; q += blockDim.x) {
        const int t = q >> 10, i = q & 1023;
        uint16_t e = 0;
        for (int l = 1; l <= 10; l++) {
            const uint32_t d = (uint32_t)((int32_t)(i >> (10 - l)) - S.first[t][l]);
            if (d < (uint32_t)S.count[t][l]) {
                e = (uint16_t)((S.perm[t][S.pidx[t][l] + (int)d] << 5) | l);
                break;
            }
        }
        S.lut[t][i] = e;
    }
    // multi-code length tables: how many whole codes the next 12 bits hold
    // (at most 4) and how many bits they take, for the group walk below
    for (int q = tid; q < S.n_groups * 4096; q += blockDim.x) {
        const int t = q >> 12, i = q & 4095;
        int used = 0, n = 0;
        while (n < 4) {
            int l = 1, got = 0;
            for (; l <= 12 - used; l++) {
                const uint32_t d = (uint32_t)((int32_t)((i >> (12 - used - l)) & ((1 << l) - 1)) - S.first[t][l]);
                if (d < (uint32_t)S.count[t][l]) { got = l; break; }
            }
            if (!got) break;
            used += got;
            n++;
        }
        S.mlut[t][i] = (uint16_t)((n << 5) | used);
    }
    __syncthreads();
    // ---- 1b. Huffman: thread 0 walks the groups once to find where each
    // starts in the stream (and where EOB is); then every thread decodes
    // whole groups from their offsets into the symbol array
    int32_t *gofs = T;                                  // group bit offsets (T is free until the LF mapping)
    uint16_t *syms = reinterpret_cast<uint16_t *>(mark);  // symbols in order (mark is free until the walkers)
    if (tid == 0) {
        AheadReader br;
        br.start(S.br);
        const int nsel = S.n_sel, alpha = S.alpha;
        int st = DEC_OK, ns = 0, ngu = 0;
        for (int g = 0; g < nsel && st == DEC_OK; g++) {
            gofs[g] = (int32_t)(br.next * 8 - br.bcnt);
            const int t = sel[g];
            int k = 0;
            if (g < nsel - 1) {
                // an encoder writes one selector per group it uses, so EOB is
                // in the last group and the others hold 50 codes: their
                // lengths only, several codes per lookup (a misplaced EOB in
                // a corrupt stream shows up in the group decode or the MTF)
                const uint16_t *ml = S.mlut[t];
                while (k < 50) {
                    if (br.bcnt < 32) br.refill();  // then the whole step needs no other check
                    const uint32_t e = ml[(uint32_t)(br.buf >> 52)];
                    const int n = (int)(e >> 5), len = (int)(e & 31);
                    if (n > 0 && n <= 50 - k && len <= br.bcnt) {
                        br.buf <<= len;
                        br.bcnt -= len;
                        k += n;
                    } else {
                        if (huff_symbol(br, S, t) < 0) { st = br.err ? DEC_TRUNC : DEC_BAD_DATA; break; }
                        k++;
                    }
                }
                continue;
            }
            for (; k < 50; k++) {
                const int sym = huff_symbol(br, S, t);
                if (sym < 0) { st = br.err ? DEC_TRUNC : DEC_BAD_DATA; break; }
                if (sym == alpha - 1) break;  // EOB
            }
            if (st != DEC_OK) break;
            if (k < 50) {
                ns = g * 50 + k + 1;
                ngu = g + 1;
                break;
            }
            st = DEC_BAD_DATA;  // no EOB
        }
        S.nsym = ns;
        S.ngroups_used = ngu;
        S.status = st;
    }
    __syncthreads();
    if (S.status != DEC_OK) {
        if (tid == 0) status[b] = S.status;
        return;
    }
    {
        const int ns = S.nsym, ngu = S.ngroups_used;
        for (int g = tid; g < ngu; g += blockDim.x) {
            BitReader br;
            br.init(D.src, D.src_len);
            const int32_t bo = gofs[g];
            br.next = bo >> 3;
            br.skip(bo & 7);
            const int t = sel[g], cnt = min(50, ns - g * 50);
            for (int k = 0; k < cnt; k++) syms[g * 50 + k] = (uint16_t)huff_symbol(br, S, t);
        }
    }
    __syncthreads();
    // ---- 1c. inverse RUNA/RUNB and MTF by segments. A segment's MTF moves
    // permute list positions whatever the list holds, so each warp first
    // finds its segment's permutation and output length (pass 1), warp 0
    // chains the lists at the segment starts and the output offsets, and
    // each warp decodes its segment from its own starting list (pass 2).
    // Segments start right after a symbol that is not a run digit, so no
    // run is split. The list lives in registers, 8 bytes per lane (lane l
    // holds positions 8l .. 8l + 7, position 8l + q in byte q of lo for q <
    // 4, of hi otherwise); moving index j to the front shifts positions
    // 0 .. j up by one byte and keeps the rest: one byte permute per word.
    {
        const int ns = S.nsym, niu = S.n_in_use, alpha = S.alpha, block_max = S.block_max;
        const int w = tid >> 5, lane = tid & 31;
        if (lane == 0) {
            const int per = (ns + kDecWarps - 1) / kDecWarps, s0 = w * per, e0 = min(ns, s0 + per);
            int p = ns;
            if (w == 0) {
                p = 0;
            } else {
                for (int q = max(s0, 1); q < e0; q++)
                    if (syms[q - 1] >= 2) { p = q; break; }
            }
            S.seg_start[w] = p;
        }
        __syncthreads();
        const int p0 = S.seg_start[w];
        int p1 = ns;
        for (int w2 = w + 1; w2 < kDecWarps; w2++)
            if (S.seg_start[w2] < ns) { p1 = S.seg_start[w2]; break; }
        for (int pass = 0; pass < 2; pass++) {
            int st = DEC_OK;
            int64_t outc = 0;
            if (p0 < ns) {
                uint32_t lo = 0, hi = 0;
                for (int q = 3; q >= 0; q--) {  // positions (pass 0) or the list at the segment start (pass 1)
                    const int a = 8 * lane + q, a4 = a + 4;
                    const uint32_t va = pass ? S.seg_list[w][a] : (uint32_t)a;
                    const uint32_t va4 = pass ? S.seg_list[w][a4] : (uint32_t)a4;
                    lo = (lo << 8) | va;
                    hi = (hi << 8) | va4;
                }
                const int64_t off = pass ? S.seg_off[w] : 0;
                int64_t run = 0, run_w = 1;
                uint32_t batch = 0;
                for (int i = p0; i < p1; i++) {
                    if (((i - p0) & 31) == 0) batch = i + lane < p1 ? syms[i + lane] : 0u;
                    const int sym = (int)__shfl_sync(LFC_FULL, batch, (i - p0) & 31);
                    if (sym <= 1) {
                        run += (int64_t)(sym + 1) * run_w;
                        run_w <<= 1;
                        if (run > block_max) { st = DEC_OVERFLOW; break; }
                        continue;
                    }
                    if (run > 0) {
                        if (pass) {
                            if (off + outc + run > S.nblock) { st = DEC_OVERFLOW; break; }
                            const uint8_t v = S.seq_to_unseq[__shfl_sync(LFC_FULL, lo, 0) & 255u];
                            for (int64_t q = lane; q < run; q += 32) L[off + outc + q] = v;
                        }
                        outc += run;
                        run = 0;
                        run_w = 1;
                    }
                    if (sym == alpha - 1) break;  // EOB
                    const int j = sym - 1;  // >= 1
                    if (j >= niu) { st = DEC_BAD_DATA; break; }
                    const uint32_t holder = __shfl_sync(LFC_FULL, (j & 4) ? hi : lo, j >> 3);
                    const uint32_t v = (holder >> (8 * (j & 3))) & 255u;
                    const uint32_t below = __shfl_up_sync(LFC_FULL, hi, 1) >> 24;  // position 8l - 1
                    const uint32_t slo = (lo << 8) | (lane == 0 ? v : below), shi = __funnelshift_l(lo, hi, 8);
                    const int cnt = min(8, max(0, j + 1 - 8 * lane));
                    const int cl = min(cnt, 4), ch = max(cnt - 4, 0);
                    lo = __byte_perm(slo, lo, 0x7654u - (0x4444u & ((1u << (4 * cl)) - 1u)));
                    hi = __byte_perm(shi, hi, 0x7654u - (0x4444u & ((1u << (4 * ch)) - 1u)));
                    if (pass) {
                        if (off + outc >= S.nblock) { st = DEC_OVERFLOW; break; }
                        if (lane == 0) L[off + outc] = S.seq_to_unseq[v];
                    }
                    outc++;
                    if (outc > block_max) { st = DEC_OVERFLOW; break; }
                }
                if (pass == 0) {  // where the moves took each position
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        S.seg_perm[w][8 * lane + q] = (uint8_t)(lo >> (8 * q));
                        S.seg_perm[w][8 * lane + 4 + q] = (uint8_t)(hi >> (8 * q));
                    }
                }
            }
            if (lane == 0) {
                S.seg_len[w] = (int32_t)(outc < INT_MAX ? outc : INT_MAX);
                S.seg_status[w] = st;
            }
            __syncthreads();
            if (pass == 0 && w == 0) {
                // lists at the segment starts and output offsets, in order
                int st0 = DEC_OK;
                for (int q = lane; q < 256; q += 32) S.seg_list[0][q] = (uint8_t)(q < niu ? q : 0);
                int64_t total = 0;
                int prev = -1;
                for (int w2 = 0; w2 < kDecWarps; w2++) {
                    if (S.seg_start[w2] >= ns) continue;
                    if (S.seg_status[w2] != DEC_OK) st0 = S.seg_status[w2];
                    if (prev >= 0) {
                        __syncwarp();
                        for (int q = lane; q < 256; q += 32) S.seg_list[w2][q] = S.seg_list[prev][S.seg_perm[prev][q]];
                    }
                    if (lane == 0) S.seg_off[w2] = (int32_t)(total < INT_MAX ? total : INT_MAX);
                    total += S.seg_len[w2];
                    prev = w2;
                }
                if (st0 == DEC_OK && (total > block_max || total > kBlockCap)) st0 = DEC_OVERFLOW;
                if (st0 == DEC_OK && S.orig >= total) st0 = DEC_BAD_ORIG;
                if (lane == 0) {
                    S.status = st0;
                    S.nblock = (int32_t)(total < INT_MAX ? total : INT_MAX);
                }
            }
            __syncthreads();
            if (S.status != DEC_OK) break;
        }
        if (tid == 0)
            for (int w2 = 0; w2 < kDecWarps; w2++)
                if (S.seg_status[w2] != DEC_OK) S.status = S.seg_status[w2];
    }
    __syncthreads();
    if (S.status != DEC_OK) {
        if (tid == 0) status[b] = S.status;
        return;
    }
    const int m = S.nblock;
    // ---- 2. LF mapping: stable counting sort of L with per-warp counters
    const int w = tid >> 5, lane = tid & 31, NW = kDecThreads / 32;
    for (int i = lane; i < 256; i += 32) S.warp_cnt[w][i] = 0;
    __syncwarp();
    const int per_w = (m + NW - 1) / NW;
    const int wa = min(m, w * per_w), we = min(m, wa + per_w);
    for (int base = wa; base < we; base += 32) {
        const int j = base + lane;
        const bool ok = j < we;
        const uint32_t c = ok ? L[j] : 0u;
        const uint32_t mm = __match_any_sync(LFC_FULL, ok ? c : 256u + lane);
        if (ok && (mm & lanemask_gt()) == 0) S.warp_cnt[w][c] += __popc(mm);
        __syncwarp();
    }
    __syncthreads();
    if (tid < 256) {
        uint32_t acc = 0;
        for (int ww = 0; ww < NW; ww++) acc += S.warp_cnt[ww][tid];
        S.C[tid] = acc;
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t acc = 0;
        for (int c = 0; c < 256; c++) { const uint32_t v = S.C[c]; S.C[c] = acc; acc += v; }
    }
    __syncthreads();
    if (tid < 256) {
        uint32_t acc = S.C[tid];
        for (int ww = 0; ww < NW; ww++) { const uint32_t v = S.warp_cnt[ww][tid]; S.warp_cnt[ww][tid] = acc; acc += v; }
    }
    __syncthreads();
    for (int base = wa; base < we; base += 32) {
        const int j = base + lane;
        const bool ok = j < we;
        const uint32_t c = ok ? L[j] : 0u;
        const uint32_t mm = __match_any_sync(LFC_FULL, ok ? c : 256u + lane);
        uint32_t before = ok ? S.warp_cnt[w][c] : 0u;
        __syncwarp();
        if (ok) {
            T[j] = (int32_t)(before + __popc(mm & lanemask_lt()));
            if ((mm & lanemask_gt()) == 0) S.warp_cnt[w][c] = before + __popc(mm);
        }
        __syncwarp();
    }
    for (int j = tid; j < m; j += blockDim.x) mark[j] = -1;
    __syncthreads();
    // ---- 3. walkers
    const int nwk = min(kWalkers, m);
    int start = -1;
    if (tid < nwk) {
        if (tid == 0) {
            start = S.orig;
        } else {
            start = (int)((int64_t)tid * m / nwk);
            if (start == S.orig) start = -1;  // orig is walker 0's row
        }
        if (start >= 0) mark[start] = tid;
    }
    __syncthreads();
    if (start >= 0) {
        int r = start, steps = 0;
        do {
            r = T[r];
            steps++;
        } while (mark[r] < 0 && steps <= m);
        S.walk_len[tid] = steps;
        S.walk_next[tid] = steps <= m ? mark[r] : -1;
    } else if (tid < kWalkers) {
        S.walk_len[tid] = 0;
        S.walk_next[tid] = -1;
    }
    __syncthreads();
    if (tid == 0) {
        int k = 0;
        int64_t pos = 0;
        int visited = 0;
        bool bad = false;
        for (int i = 0; i < kWalkers; i++) S.walk_pos[i] = -1;
        while (pos < m) {
            if (k < 0 || k >= kWalkers || S.walk_pos[k] >= 0 || S.walk_len[k] <= 0) { bad = true; break; }
            S.walk_pos[k] = pos;
            pos += S.walk_len[k];
            visited++;
            k = S.walk_next[k];
        }
        if (bad || pos != m || k != 0) S.status = DEC_BAD_WALK;
    }
    __syncthreads();
    if (S.status != DEC_OK) {
        if (tid == 0) status[b] = S.status;
        return;
    }
    if (start >= 0 && S.walk_pos[tid] >= 0) {
        int r = start;
        const int64_t p0 = S.walk_pos[tid];
        for (int s = 0; s < S.walk_len[tid]; s++) {
            blk[m - 1 - (p0 + s)] = L[r];
            r = T[r];
        }
    }
    __syncthreads();
    // ---- 4. inverse RLE1, then CRC. A position q is a sync point when
    // bytes q-2 and q-1 differ and bytes q-5 .. q-2 are not all equal: byte
    // q-1 is then a literal (a count byte follows four equal literals) that
    // starts a run, so decoding can start at q from (run 1, last = byte
    // q-1). Every thread takes the first sync point of its chunk (thread 0:
    // position 0, fresh) and decodes up to the next thread's: once to count
    // its output bytes, once to write them at their prefix.
    {
        const int nth = blockDim.x;
        const int ch = max(8, (m + nth - 1) / nth);
        const int s0 = tid * ch, e0 = min(m, s0 + ch);
        int p = m;  // this thread's segment start, m: none in its chunk
        if (s0 < m) {
            if (tid == 0) {
                p = 0;
            } else {
                for (int q = max(s0, 5); q < e0; q++) {
                    const uint8_t b1 = blk[q - 1], b2 = blk[q - 2];
                    if (b1 != b2 && !(blk[q - 5] == b2 && blk[q - 4] == b2 && blk[q - 3] == b2)) { p = q; break; }
                }
            }
        }
        S.walk_len[tid] = p;
        __syncthreads();
        int end = m;  // the next segment start after this one
        if (p < m)
            for (int t2 = tid + 1; t2 < nth; t2++)
                if (S.walk_len[t2] < m) { end = S.walk_len[t2]; break; }
        int cnt = 0, st = DEC_OK;
        for (int pass = 0; pass < 2; pass++) {
            int off = 0;
            if (pass == 1) {
                int total = 0;
                off = block_excl_sum<int>(cnt, S.scan_sh, &total);
                if (total != D.expect) st = DEC_BAD_LEN;
                if (__syncthreads_or(st != DEC_OK)) break;
            }
            if (p < m) {
                int o = 0, same = tid == 0 ? 0 : 1, last = tid == 0 ? -1 : (int)blk[p - 1];
                for (int i = p; i < end; i++) {
                    const uint8_t v = blk[i];
                    if (pass) D.dst[off + o] = v;
                    o++;
                    same = ((int)v == last) ? same + 1 : 1;
                    last = v;
                    if (same == 4) {
                        if (i + 1 >= m) { st = DEC_BAD_DATA; break; }
                        const int extra = blk[++i];
                        if (pass && off + o + extra > D.expect) { st = DEC_BAD_LEN; break; }
                        if (pass)
                            for (int q = 0; q < extra; q++) D.dst[off + o + q] = v;
                        o += extra;
                        same = 0;
                        last = -1;
                    }
                }
                cnt = o;
            }
            if (__syncthreads_or(st != DEC_OK)) break;
        }
        if (tid == 0) {
            S.status = DEC_OK;
            S.out_len = D.expect;
        }
        __syncthreads();
        if (st != DEC_OK) S.status = st;  // any failing thread (benign race: all write an error code)
    }
    __syncthreads();
    if (S.status != DEC_OK) {
        if (tid == 0) status[b] = S.status;
        return;
    }
    const int n = S.out_len;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int a = min(n, tid * per), e = min(n, a + per);
    uint32_t r = 0;
    for (int i = a; i < e; i++) r = (r << 8) ^ S.crc_tab[(r >> 24) ^ D.dst[i]];
    if (e > a) r = gf_mul(r, xpow8((uint64_t)(n - e)));
    for (int o = 16; o > 0; o >>= 1) r ^= __shfl_xor_sync(LFC_FULL, r, o);
    if (lane == 0) S.red[w] = r;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int i = 0; i < NW; i++) t ^= S.red[i];
        t ^= gf_mul(0xFFFFFFFFu, xpow8((uint64_t)n));
        status[b] = (~t == S.stored_crc) ? DEC_OK : DEC_BAD_CRC;
    }
}

// ------------------------------------------------------ inverse predictor
__device__ __forceinline__ int32_t as_s16(uint32_t v) { return (int32_t)(int16_t)(uint16_t)v; }
__device__ __forceinline__ uint32_t unzig(uint32_t z) { return (uint32_t)(((z >> 1) ^ (0u - (z & 1u))) & 0xFFFFu); }

__device__ __forceinline__ int32_t jp(int f, int32_t A, int32_t B, int32_t C) {
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
__device__ __forceinline__ int32_t gp(int f, int row, int col, int32_t A, int32_t B, int32_t C) {
    if (row == 0) return col == 0 ? 0 : A;
    if (col == 0) return B;
    return jp(f, A, B, C);
}

struct InvFrame {
    const uint16_t *Z;      // symbol stream (stream order)
    const uint16_t *prev;   // previous raw frame or nullptr
    uint16_t *X;            // output frame
    int32_t *E;             // int32 scratch field (W*H)
    int32_t W, H, p, id;
};

__device__ __forceinline__ size_t stream_index(const InvFrame &F, int y, int x) {
    if (!((F.id >> 6) & 1)) return (size_t)y * F.W + x;
    const int Nx = F.W / F.p, Ny = F.H / F.p;
    const int t = y / F.p, v = y % F.p, s = x / F.p, u = x % F.p;
    return (size_t)(v * Ny + t) * F.W + (size_t)u * Nx + s;
}

// Residual field e at every pixel (raw for f == 0 without temporal).
__global__ void inv_residual_kernel(InvFrame F) {
    const int64_t n = (int64_t)F.W * F.H;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(k / F.W), x = (int)(k % F.W);
        const size_t si = stream_index(F, y, x);
        // planar layout: high bytes of all symbols, then their low bytes
        const uint8_t *Z8 = reinterpret_cast<const uint8_t *>(F.Z);
        const uint32_t z = id_planar(F.id) ? ((uint32_t)Z8[si] << 8) | Z8[(size_t)n + si] : F.Z[si];
        const int f = id_f(F.id);
        const bool tmp = id_tmp(F.id);
        F.E[k] = (f == 0 && !tmp) ? (int32_t)z : as_s16(unzig(z));
    }
}

// Inter-lenslet inverse over the view grid of every (u, v): one CTA per
// view restores its Ny x Nx grid by anti-diagonals (cell (t, s) needs the
// cells left, above and above-left, all on the two previous diagonals), one
// thread per cell of a diagonal. signed_out: keep the result as signed
// 16-bit (phase stage / temporal fields).
__global__ void __launch_bounds__(128) inv_inter_kernel(InvFrame F, int signed_field) {
    const int p = F.p, Nx = F.W / p, Ny = F.H / p;
    const int view = blockIdx.x;
    const int v = view / p, u = view % p;
    const int f = id_f(F.id);
    for (int d = 0; d < Nx + Ny - 1; d++) {
        const int t_lo = max(0, d - (Nx - 1)), t_hi = min(Ny - 1, d);
        for (int t = t_lo + (int)threadIdx.x; t <= t_hi; t += blockDim.x) {
            const int s = d - t;
            const size_t k = (size_t)(t * p + v) * F.W + s * p + u;
            const int32_t A = s > 0 ? F.E[k - p] : 0;
            const int32_t B = t > 0 ? F.E[k - (size_t)p * F.W] : 0;
            const int32_t C = (s > 0 && t > 0) ? F.E[k - (size_t)p * F.W - p] : 0;
            const uint32_t val = ((uint32_t)F.E[k] + (uint32_t)gp(f, t, s, A, B, C)) & 0xFFFFu;
            F.E[k] = signed_field ? as_s16(val) : (int32_t)val;
        }
        __syncthreads();
    }
}

// Intra-lenslet inverse: one thread per lenslet, raster order inside it.
__global__ void inv_intra_kernel(InvFrame F, int signed_field) {
    const int p = F.p, Nx = F.W / p, Ny = F.H / p;
    const int lens = blockIdx.x * blockDim.x + threadIdx.x;
    if (lens >= Nx * Ny) return;
    const int t = lens / Nx, s = lens % Nx;
    const int f = id_f(F.id);
    for (int v = 0; v < p; v++) {
        for (int u = 0; u < p; u++) {
            const size_t k = (size_t)(t * p + v) * F.W + s * p + u;
            const int32_t A = u > 0 ? F.E[k - 1] : 0;
            const int32_t B = v > 0 ? F.E[k - F.W] : 0;
            const int32_t C = (u > 0 && v > 0) ? F.E[k - F.W - 1] : 0;
            const uint32_t val = ((uint32_t)F.E[k] + (uint32_t)gp(f, v, u, A, B, C)) & 0xFFFFu;
            F.E[k] = signed_field ? as_s16(val) : (int32_t)val;
        }
    }
}

// Base field -> raw counts (adds the previous frame for temporal ids).
__global__ void inv_finish_kernel(InvFrame F) {
    const int64_t n = (int64_t)F.W * F.H;
    const bool tmp = (F.id >> 7) & 1;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = (uint32_t)F.E[k];
        if (tmp) v += F.prev[k];
        F.X[k] = (uint16_t)(v & 0xFFFFu);
    }
}

size_t decode_smem_bytes() { return sizeof(DecShared); }

cudaError_t launch_bzip2_decode(lfc_plan P, const void *d_blocks, int nblocks, int32_t *d_status) {
    Workspace &ws = P->ws;
    const size_t smem = sizeof(DecShared);
    cudaError_t e = cudaFuncSetAttribute(bzip2_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    bzip2_decode_kernel<<<nblocks, kDecThreads, smem, P->stream>>>(reinterpret_cast<const DecBlock *>(d_blocks), d_status,
                                                                  ws.sel, ws.bwt, ws.sa, ws.sa2, ws.rle);
    count_launches(P, 1);
    return cudaGetLastError();
}

cudaError_t launch_inverse_predict(lfc_plan P, const uint16_t *Z, const uint16_t *prev, uint16_t *X, int32_t *E,
                                   int W, int H, int p, int id) {
    InvFrame F{Z, prev, X, E, W, H, p, id};
    cudaStream_t s = P->stream;
    const int f = id_f(id), dom = id_dom(id);
    const bool tmp = id_tmp(id);
    inv_residual_kernel<<<1216, 256, 0, s>>>(F);
    int launches = 2;
    if (f != 0) {
        const int nl = (W / p) * (H / p), nv = p * p;
        if (dom == 0) {
            inv_intra_kernel<<<(nl + 127) / 128, 128, 0, s>>>(F, tmp ? 1 : 0);
            launches++;
        } else if (dom == 1) {
            inv_inter_kernel<<<nv, 128, 0, s>>>(F, tmp ? 1 : 0);
            launches++;
        } else {
            inv_inter_kernel<<<nv, 128, 0, s>>>(F, 1);
            inv_intra_kernel<<<(nl + 127) / 128, 128, 0, s>>>(F, tmp ? 1 : 0);
            launches += 2;
        }
    }
    inv_finish_kernel<<<1216, 256, 0, s>>>(F);
    count_launches(P, launches);
    return cudaGetLastError();
}

}  // namespace lfc

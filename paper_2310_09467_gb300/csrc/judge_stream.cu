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
// 2. chain_hist_kernel: one CTA (10 warps) per segment of a candidate
//    stream, one warp per range (at most the tuned 16-256 KB, evened out per
//    launch), one lane per 32nd of the range walking it byte by byte (see
//    below); the lanes' sub-ranges are stitched per warp, the ranges per CTA
//    and the CTAs by the fixup kernel.
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

// Division by a per-CTA constant d (1 <= d < 2^16) as a multiply-high by
// m = ceil(2^32 / d): floor(n * m / 2^32) = floor(n / d) exactly for
// n < 2^16, because n * (m d - 2^32) < 2^32. Every index divided here (tile
// pixels, runs, views) stays below 2^16.
struct DivU16 {
    uint64_t m;
    uint32_t d;
    __device__ explicit DivU16(uint32_t d_) : m(((1ull << 32) + d_ - 1) / d_), d(d_) {}
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return (uint32_t)(((uint64_t)n * m) >> 32); }
    __device__ __forceinline__ uint32_t mod(uint32_t n) const { return n - div(n) * d; }
};

// nslots bounds both the residual fields (f with an intra or phase-space
// candidate) and the symbol planes (f with an inter or phase-space candidate).
size_t emit_all_smem_bytes(int p, int ts, int nslots) {
    const size_t cells = (size_t)(2 * p) * (size_t)((ts + 1) * p);
    const size_t outpx = (size_t)p * (size_t)(ts * p);
    return cells * 2 * (size_t)(1 + nslots) + outpx * 2 * (size_t)(nslots > 0 ? nslots : 1) + 256;
}

// grid (tiles, frames, kind); kind 0 = raw base field, 1 = temporal difference.
// Symbols do not depend on the ordering, only their positions do: per
// predictor function f, the intra / inter / phase-space symbols of the
// tile's pixels are computed once into shared memory (thread = pixel column,
// p rows each), then every candidate of that f is written from there in
// its ordering, consecutive threads on consecutive output positions.
// PL: the candidate set holds planar-layout ids (otherwise their stores
// compile away).
template <int kind, bool PL>
__device__ __forceinline__ void emit_all_body(const JudgeFrame *__restrict__ frames, const uint8_t *__restrict__ cand,
                                              uint8_t *__restrict__ cstream, int64_t cslot, int kmax, int TS,
                                              uint8_t *esm, int16_t (*slot_of)[3][2][2], int8_t *eslot_of) {
    const int fi = blockIdx.y;
    const JudgeFrame &J = frames[fi];
    const FrameDev F = J.F;
    if (kind == 1 && F.prev == nullptr) return;
    const int p = F.p, Nx = F.Nx, Ny = F.Ny, W = F.W;
    const int tiles_s = (Nx + TS - 1) / TS;
    if ((int)blockIdx.x >= Ny * tiles_s) return;
    const int t = blockIdx.x / tiles_s, s0 = (blockIdx.x % tiles_s) * TS, ns = min(TS, Nx - s0);
    const int TR = 2 * p, TC = (TS + 1) * p, ncols = (ns + 1) * p;
    const int cells = TR * TC;
    const int nco = ns * p, npx = p * nco;  // output columns and pixels of the tile
    uint32_t fset = 0, fany = 0;
    int nc = 0;
    for (int k = 0; k < J.K; k++) {
        const int id = cand[J.cand_off + k];
        if (((id >> 7) & 1) != kind || !cand_on(J, id)) continue;
        nc++;
        const int f = id_f(id), dom = id_dom(id);
        fany |= 1u << f;
        if (f && dom != 1) fset |= 1u << f;
    }
    if (nc == 0) return;
    const int nslots = __popc(fset);
    uint16_t *Fb = reinterpret_cast<uint16_t *>(esm);
    int16_t *E = reinterpret_cast<int16_t *>(esm) + cells;
    uint16_t *Sy = reinterpret_cast<uint16_t *>(E + (size_t)nslots * cells);  // [3][npx]
    if (threadIdx.x == 0) {
        for (int i = 0; i < 96; i++) (&slot_of[0][0][0][0])[i] = -1;
        for (int f = 0; f < 8; f++) eslot_of[f] = (int8_t)__popc(fset & ((1u << f) - 1u));
        for (int k = 0; k < J.K; k++) {
            const int id = cand[J.cand_off + k];
            if (((id >> 7) & 1) != kind || !cand_on(J, id)) continue;
            slot_of[id_f(id)][id_dom(id)][id_ord(id)][id_planar(id)] = (int16_t)k;
        }
    }
    const DivU16 div_p((uint32_t)p);
    const int y0 = (t - 1) * p, x0 = (s0 - 1) * p;
    // the tile's rows y0 .. y0 + TR - 1, columns x0 .. x0 + ncols - 1 (zero
    // outside the frame): with 16-byte aligned rows, as 16-byte loads of 8
    // pixels from the multiple of 8 at or below x0 (a chunk never straddles
    // column 0 or the row end); otherwise pixel by pixel
    const bool vec = (W % 8) == 0 && (reinterpret_cast<uintptr_t>(F.X) & 15) == 0 &&
                     (!kind || (reinterpret_cast<uintptr_t>(F.prev) & 15) == 0);
    if (vec) {
        const int xa0 = x0 >= 0 ? (x0 & ~7) : -((7 - x0) & ~7);
        const int nch = (x0 + ncols - xa0 + 7) >> 3;
        for (int q = threadIdx.x; q < TR * nch; q += blockDim.x) {
            const int ly = q / nch, xa = xa0 + 8 * (q - ly * nch), y = y0 + ly;
            uint4 a = make_uint4(0, 0, 0, 0), b = a;
            if (y >= 0 && xa >= 0) {
                a = __ldg(reinterpret_cast<const uint4 *>(F.X + (size_t)y * W + xa));
                if (kind) b = __ldg(reinterpret_cast<const uint4 *>(F.prev + (size_t)y * W + xa));
            }
            const uint32_t aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int lx = xa + j - x0;
                if (lx < 0 || lx >= ncols) continue;
                uint32_t v = (aw[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
                if (kind) v = (v - ((bw[j >> 1] >> (16 * (j & 1))) & 0xFFFFu)) & 0xFFFFu;
                Fb[ly * TC + lx] = (uint16_t)v;
            }
        }
    } else {
        for (int lx = threadIdx.x; lx < ncols; lx += blockDim.x) {  // column per thread, rows in a loop
            const int x = x0 + lx;
            for (int ly = 0; ly < TR; ly++) {
                const int y = y0 + ly;
                uint32_t v = 0;
                if (y >= 0 && x >= 0) {
                    const size_t k = (size_t)y * W + x;
                    v = __ldg(F.X + k);
                    if (kind) v = (v - (uint32_t)__ldg(F.prev + k)) & 0xFFFFu;
                }
                Fb[ly * TC + lx] = (uint16_t)v;
            }
        }
    }
    __syncthreads();
#define FVAL(idx) (kind ? (int32_t)(int16_t)Fb[idx] : (int32_t)Fb[idx])  // kind is a template constant
    // intra residual fields (signed 16-bit) for every f in use
    for (int lx = threadIdx.x; lx < ncols; lx += blockDim.x) {
        const int u = (int)div_p.mod((uint32_t)lx);
        for (int ly = 0; ly < TR; ly++) {
            const int v = ly < p ? ly : ly - p;  // TR = 2p rows
            const int idx = ly * TC + lx;
            const int32_t Xv = FVAL(idx);
            const int32_t A = u > 0 ? FVAL(idx - 1) : 0;
            const int32_t B = v > 0 ? FVAL(idx - TC) : 0;
            const int32_t C = (u > 0 && v > 0) ? FVAL(idx - TC - 1) : 0;
#pragma unroll
            for (int f = 1; f < 8; f++)
                if (fset & (1u << f)) E[(size_t)eslot_of[f] * cells + idx] = (int16_t)(Xv - g_pred(f, v, u, A, B, C));
        }
    }
    __syncthreads();
    uint8_t *base8 = cstream + (size_t)fi * kmax * (size_t)cslot;
    uint16_t *base = reinterpret_cast<uint16_t *>(base8);
    const size_t cslot16 = (size_t)cslot / 2;
    const size_t nsym = (size_t)W * F.H;  // a planar stream's low bytes start here
    // view-major write-out: thread j -> (u, si) = (j / ns, j % ns), rows v
    const DivU16 div_ns((uint32_t)ns);
    const int vm_j = threadIdx.x, vm_u = (int)div_ns.div((uint32_t)vm_j), vm_si = vm_j - vm_u * ns;
    // vector stores when every run start is aligned (slots are 256-byte aligned;
    // raw rows: W and the tile's first column multiples of 8 pixels keep every
    // 8-pixel run on a 16-byte boundary, and its planar bytes on 8-byte ones)
    const bool raw8 = (W % 8) == 0 && ((s0 * p) % 8) == 0 && (nco % 8) == 0;
    const bool raw2 = (W % 2) == 0 && ((s0 * p) % 2) == 0 && (nco % 2) == 0;
    const bool vm8 = (ns % 8) == 0 && (W % 8) == 0 && (Nx % 8) == 0 && (s0 % 8) == 0;
    const DivU16 div_h((uint32_t)max(nco >> 1, 1)), div_h8((uint32_t)max(nco >> 3, 1)), div_hn((uint32_t)max(ns >> 3, 1));
    // 8 symbols (4 words, two per word) as 8 high bytes and 8 low bytes
    auto put8 = [&](uint8_t *hi, const uint4 &o) {
        *reinterpret_cast<uint2 *>(hi) = make_uint2(__byte_perm(o.x, o.y, 0x7531), __byte_perm(o.z, o.w, 0x7531));
        *reinterpret_cast<uint2 *>(hi + nsym) = make_uint2(__byte_perm(o.x, o.y, 0x6420), __byte_perm(o.z, o.w, 0x6420));
    };
    auto put1 = [&](uint8_t *hi, uint32_t v) {
        hi[0] = (uint8_t)(v >> 8);
        hi[nsym] = (uint8_t)v;
    };
    // Writes the symbols get(r, c) of the tile's output pixels (row r of the
    // lenslet row, column c) in raw order to candidate k0 ((lo, hi) layout)
    // and k0p (planar layout), and in view-major order (view v = r, u = c mod
    // p, lenslet s0 + c / p) to k1 and k1p; consecutive threads on
    // consecutive output positions, every symbol computed once.
    auto write_both = [&](int k0, int k1, int k0p, int k1p, auto get) {
        if (k0 >= 0 || k0p >= 0) {
            const size_t i0 = (size_t)(t * p) * W + (size_t)s0 * p;  // symbol index of the tile's first pixel
            uint16_t *dst = k0 >= 0 ? base + (size_t)k0 * cslot16 + i0 : nullptr;
            uint8_t *dsp = PL && k0p >= 0 ? base8 + (size_t)k0p * cslot + i0 : nullptr;
            if (raw8) {  // 8 pixels per 16-byte store
                const int h = nco >> 3;
                for (int q = threadIdx.x; q < p * h; q += blockDim.x) {
                    const int r = (int)div_h8.div((uint32_t)q), c8 = 8 * (q - r * h);
                    uint4 o;
                    o.x = (uint32_t)get(r, c8) | ((uint32_t)get(r, c8 + 1) << 16);
                    o.y = (uint32_t)get(r, c8 + 2) | ((uint32_t)get(r, c8 + 3) << 16);
                    o.z = (uint32_t)get(r, c8 + 4) | ((uint32_t)get(r, c8 + 5) << 16);
                    o.w = (uint32_t)get(r, c8 + 6) | ((uint32_t)get(r, c8 + 7) << 16);
                    if (dst) *reinterpret_cast<uint4 *>(dst + (size_t)r * W + c8) = o;
                    if (dsp) put8(dsp + (size_t)r * W + c8, o);
                }
            } else if (raw2) {
                const int h = nco >> 1;
                for (int q = threadIdx.x; q < p * h; q += blockDim.x) {
                    const int r = (int)div_h.div((uint32_t)q), c2 = 2 * (q - r * h);
                    const uint32_t a = get(r, c2), b = get(r, c2 + 1);
                    if (dst) *reinterpret_cast<uint32_t *>(dst + (size_t)r * W + c2) = a | (b << 16);
                    if (dsp) {
                        *reinterpret_cast<uint16_t *>(dsp + (size_t)r * W + c2) = (uint16_t)((a >> 8) | (b & 0xFF00u));
                        *reinterpret_cast<uint16_t *>(dsp + nsym + (size_t)r * W + c2) = (uint16_t)((a & 0xFFu) | ((b & 0xFFu) << 8));
                    }
                }
            } else {
                for (int r = 0; r < p; r++)
                    for (int c = threadIdx.x; c < nco; c += blockDim.x) {
                        const uint32_t v = get(r, c);
                        if (dst) dst[(size_t)r * W + c] = (uint16_t)v;
                        if (dsp) put1(dsp + (size_t)r * W + c, v);
                    }
            }
        }
        if (k1 >= 0 || k1p >= 0) {
            const size_t i1 = (size_t)t * W + s0;
            uint16_t *dst = k1 >= 0 ? base + (size_t)k1 * cslot16 + i1 : nullptr;
            uint8_t *dsp = PL && k1p >= 0 ? base8 + (size_t)k1p * cslot + i1 : nullptr;
            if (vm8) {
                const int hn = ns >> 3, items = p * p * hn;
                for (int q = threadIdx.x; q < items; q += blockDim.x) {
                    const int vu = (int)div_hn.div((uint32_t)q), hh = q - vu * hn;
                    const int v = (int)div_p.div((uint32_t)vu), u = vu - v * p;
                    const int c = 8 * hh * p + u;
                    uint4 o;
                    o.x = (uint32_t)get(v, c) | ((uint32_t)get(v, c + p) << 16);
                    o.y = (uint32_t)get(v, c + 2 * p) | ((uint32_t)get(v, c + 3 * p) << 16);
                    o.z = (uint32_t)get(v, c + 4 * p) | ((uint32_t)get(v, c + 5 * p) << 16);
                    o.w = (uint32_t)get(v, c + 6 * p) | ((uint32_t)get(v, c + 7 * p) << 16);
                    const size_t e = (size_t)v * Ny * W + (size_t)u * Nx + 8 * hh;
                    if (dst) *reinterpret_cast<uint4 *>(dst + e) = o;
                    if (dsp) put8(dsp + e, o);
                }
            } else if (p * ns <= (int)blockDim.x) {
                if (vm_j < p * ns)
                    for (int v = 0; v < p; v++) {
                        const uint32_t val = get(v, vm_si * p + vm_u);
                        const size_t e = (size_t)v * Ny * W + (size_t)vm_u * Nx + vm_si;
                        if (dst) dst[e] = (uint16_t)val;
                        if (dsp) put1(dsp + e, val);
                    }
            } else {
                for (int v = 0; v < p; v++)
                    for (int j = threadIdx.x; j < p * ns; j += blockDim.x) {
                        const int u = (int)div_ns.div((uint32_t)j), si = j - u * ns;
                        const uint32_t val = get(v, si * p + u);
                        const size_t e = (size_t)v * Ny * W + (size_t)u * Nx + si;
                        if (dst) dst[e] = (uint16_t)val;
                        if (dsp) put1(dsp + e, val);
                    }
            }
        }
    };
    // raw candidates (no predictor) and intra-lenslet candidates straight from
    // the staged frame and the residual fields
    if (fany & 1u)
        write_both(slot_of[0][0][0][0], slot_of[0][0][1][0], slot_of[0][0][0][1], slot_of[0][0][1][1], [&](int r, int c) -> uint16_t {
            const int32_t Xv = FVAL((p + r) * TC + p + c);
            return kind ? zz16(Xv) : (uint16_t)Xv;
        });
#pragma unroll
    for (int f = 1; f < 8; f++) {
        if (!((fset >> f) & 1u) || (slot_of[f][0][0][0] < 0 && slot_of[f][0][1][0] < 0 && slot_of[f][0][0][1] < 0 &&
                                    slot_of[f][0][1][1] < 0))
            continue;
        const int16_t *Ef = E + (size_t)eslot_of[f] * cells;
        write_both(slot_of[f][0][0][0], slot_of[f][0][1][0], slot_of[f][0][0][1], slot_of[f][0][1][1],
                   [&](int r, int c) -> uint16_t { return zz16(Ef[(p + r) * TC + p + c]); });
    }
    // inter-lenslet candidates of every f in one pass over the pixels, then
    // the phase-space ones: symbols into planes of Sy, then written out
    for (int dom = 1; dom <= 2; dom++) {
        uint32_t fm = 0;
        int plane[8];
        int np = 0;
#pragma unroll
        for (int f = 1; f < 8; f++) {
            plane[f] = -1;
            if ((fany >> f) & 1u && (slot_of[f][dom][0][0] >= 0 || slot_of[f][dom][1][0] >= 0 ||
                                     slot_of[f][dom][0][1] >= 0 || slot_of[f][dom][1][1] >= 0)) {
                fm |= 1u << f;
                plane[f] = np++;
            }
        }
        if (!fm) continue;
        for (int c = threadIdx.x; c < nco; c += blockDim.x) {
            const int sc = (int)div_p.div((uint32_t)c);
            const int lx = p + c, s = s0 + sc;
            for (int r = 0; r < p; r++) {
                const int idx = (p + r) * TC + lx, q = r * nco + c;
                if (dom == 1) {
                    const int32_t Xv = FVAL(idx);
                    const int32_t XA = s > 0 ? FVAL(idx - p) : 0;
                    const int32_t XB = t > 0 ? FVAL(idx - p * TC) : 0;
                    const int32_t XC = (s > 0 && t > 0) ? FVAL(idx - p * TC - p) : 0;
#pragma unroll
                    for (int f = 1; f < 8; f++)
                        if ((fm >> f) & 1u) Sy[(size_t)plane[f] * npx + q] = zz16(Xv - g_pred(f, t, s, XA, XB, XC));
                } else {
#pragma unroll
                    for (int f = 1; f < 8; f++) {
                        if (!((fm >> f) & 1u)) continue;
                        const int16_t *Ef = E + (size_t)eslot_of[f] * cells;
                        const int32_t e = Ef[idx];
                        const int32_t eA = s > 0 ? Ef[idx - p] : 0;
                        const int32_t eB = t > 0 ? Ef[idx - p * TC] : 0;
                        const int32_t eC = (s > 0 && t > 0) ? Ef[idx - p * TC - p] : 0;
                        Sy[(size_t)plane[f] * npx + q] = zz16(e - g_pred(f, t, s, eA, eB, eC));
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int f = 1; f < 8; f++) {
            if (!((fm >> f) & 1u)) continue;
            const uint16_t *src = Sy + (size_t)plane[f] * npx;
            write_both(slot_of[f][dom][0][0], slot_of[f][dom][1][0], slot_of[f][dom][0][1], slot_of[f][dom][1][1],
                       [&](int r, int c) -> uint16_t { return src[r * nco + c]; });
        }
        __syncthreads();
    }
#undef FVAL
}

template <bool PL>
__global__ void __launch_bounds__(kEmitThreads) emit_all_kernel(const JudgeFrame *__restrict__ frames,
                                                                const uint8_t *__restrict__ cand, uint8_t *__restrict__ cstream,
                                                                int64_t cslot, int kmax, int TS) {
    extern __shared__ __align__(16) uint8_t esm[];
    __shared__ int16_t slot_of[8][3][2][2];  // candidate index for (f, domain, ordering, layout), -1 if absent
    __shared__ int8_t eslot_of[8];        // intra residual field of f
    if (blockIdx.z == 0) emit_all_body<0, PL>(frames, cand, cstream, cslot, kmax, TS, esm, slot_of, eslot_of);
    else emit_all_body<1, PL>(frames, cand, cstream, cslot, kmax, TS, esm, slot_of, eslot_of);
}

// ------------------------------------------------------ pair-chain histogram
// The judge-BWT's last column lists, bucket by bucket (first byte b), the
// predecessors of b's occurrences in stream order, so its bigram histogram
// counts the pairs (pred of one occurrence of b, pred of the next one), plus
// the pairs across bucket boundaries (fixup kernel).
//
// A warp takes a contiguous range of a candidate stream and gives each lane
// one 32nd of it. A lane walks its sub-range byte by byte with a private
// table over the 256 byte values: entry (b, lane) is 16 bits, the
// predecessor p of the last occurrence of b so far, kept as p * 128 so that
// a pair's hot-corner index is one addition (0xFFFF before the first
// occurrence), in the word (b / 2) * 32 + lane, half b % 2, so each lane
// stays in its own bank whatever the bytes. The predecessor of a lane's
// first occurrence of b (written once per value, read once when stitching)
// goes to a global scratch of the CTA's SM: the table's shared memory admits
// one CTA per SM. 32 bytes at a time, all table entries are read and
// rewritten first (a load only waits on the lane's own earlier stores), then
// the pairs are counted from the entries read. Afterwards the lanes' tables
// are stitched in lane order into the warp's, the warps' in order into the
// CTA's, the CTAs' by the fixup kernel. Pairs (x, y) with x, y < kHot are
// counted in shared memory: (0, 0) in the lane's own slot (no two lanes of a
// warp share its bank), added to bin (0, 0) at the end, the others in the
// hot corner; all other pairs go with fire-and-forget atomics to the
// L2-resident histogram. Every byte issues exactly one shared atomic (+0 to
// the lane's slot when its pair is counted elsewhere or it has none), so the
// walk has no branch on the data.
constexpr int kChainWarps = 10;
constexpr int kChainThreads = kChainWarps * 32;
constexpr int kHotShift = 7;                    // table entries hold p << kHotShift
constexpr int kHot = 1 << kHotShift;            // hot corner side
constexpr int kChainTab = 128 * 32;    // table words of a warp (two 16-bit entries each)
constexpr int kChainFirst = 256 * 32;  // first-predecessor bytes of a warp, [b][lane]
constexpr uint32_t kNoPred = 0xFFFF;

size_t chain_smem_bytes() { return (size_t)(kHot * kHot + 32) * 4 + (size_t)kChainWarps * kChainTab * 4; }
constexpr uint32_t kHotBins = kHot * kHot;  // (p * kHot + a) for p, a < kHot; then one slot per lane
int64_t chain_seg_bytes(int range_bytes) { return (int64_t)kChainWarps * range_bytes; }
size_t chain_first_bytes(int nsm) { return (size_t)nsm * kChainWarps * kChainFirst; }

__global__ void nsmid_kernel(int32_t *out) {
    uint32_t v;
    asm("mov.u32 %0, %%nsmid;" : "=r"(v));
    *out = (int32_t)v;
}

cudaError_t query_nsmid(cudaStream_t s, int *nsm) {
    int32_t *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int32_t));
    if (e != cudaSuccess) return e;
    nsmid_kernel<<<1, 1, 0, s>>>(d);
    int32_t h = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    *nsm = h;
    return e;
}

__device__ __forceinline__ int find_frame_s(const JudgeFrame *fr, int n, int64_t cta) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fr[mid].cta_base <= cta) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Count the pair (p, a) of a chain: e the table entry of the previous
// occurrence (p << kHotShift, kNoPred: none, nothing counted), a the predecessor of
// this one. (0, 0) adds 1 to the lane's own slot, another pair of bytes
// below kHot adds 1 to its hot-corner bin, every other lane adds 0 to its
// slot; pairs outside the corner go to the global histogram.
__device__ __forceinline__ void chain_count(uint32_t e, uint32_t a, uint32_t *hot, uint32_t *ghist, uint32_t slot) {
    const uint32_t t = e + a;                              // p * kHot + a
    const bool in_hot = (e | (a << kHotShift)) < kHotBins;  // p < kHot and a < kHot (never for kNoPred)
    atomicAdd(&hot[(in_hot && t != 0u) ? t : slot], in_hot ? 1u : 0u);
    if (e != kNoPred && !in_hot) atomicAdd(&ghist[(e << (8 - kHotShift)) | a], 1u);  // (p << 8) | a
}

__device__ __forceinline__ uint32_t byte_of(const uint32_t (&w)[8], int i) {
    return __byte_perm(w[i >> 2], 0u, 0x4440u | (uint32_t)(i & 3));
}

// Entry b of a lane's table; tl = the table + lane (words).
__device__ __forceinline__ uint16_t *chain_entry(uint32_t *tl, uint32_t b) {
    return reinterpret_cast<uint16_t *>(tl + (b >> 1) * 32) + (b & 1);
}

// 32 stream bytes (w little-endian) after the byte prev; fl = the lane's
// first-predecessor column (byte b * 32).
__device__ __forceinline__ void chain_walk32(const uint32_t (&w)[8], uint32_t &prev, uint32_t *tl, uint8_t *fl,
                                             uint32_t *hot, uint32_t *ghist, uint32_t slot) {
    uint32_t e[32];
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const uint32_t b = byte_of(w, i);
        const uint32_t a = i == 0 ? prev : byte_of(w, i - 1);
        uint16_t *en = chain_entry(tl, b);
        e[i] = *en;
        *en = (uint16_t)(a << kHotShift);
    }
#pragma unroll
    for (int i = 0; i < 32; i++) {
        const uint32_t b = byte_of(w, i);
        const uint32_t a = i == 0 ? prev : byte_of(w, i - 1);
        if (e[i] == kNoPred) fl[b * 32] = (uint8_t)a;
        chain_count(e[i], a, hot, ghist, slot);
    }
    prev = byte_of(w, 31);
}

__global__ void __launch_bounds__(kChainThreads, 1)
chain_hist_kernel(const JudgeFrame *__restrict__ frames, int nframes, const uint8_t *__restrict__ cand,
                  const uint8_t *__restrict__ cstream, int64_t cslot, int kmax, uint32_t *__restrict__ hist,
                  uint16_t *__restrict__ summ, int range_bytes, uint8_t *__restrict__ first_all, int nsm) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *hot = reinterpret_cast<uint32_t *>(smem);                 // [kHot][kHot] + 32 dummies
    uint32_t *tab_all = hot + kHot * kHot + 32;                          // [warps][128][32]
    const int fi = find_frame_s(frames, nframes, blockIdx.x);
    const JudgeFrame &J = frames[fi];
    const int64_t local = (int64_t)blockIdx.x - J.cta_base;
    const int ci = (int)(local / J.segs), seg = (int)(local % J.segs);
    if (!cand_on(J, cand[J.cand_off + ci])) return;  // not proposed: no stream, no histogram
    const uint8_t *S = cstream + ((size_t)fi * kmax + ci) * (size_t)cslot;
    uint32_t *ghist = hist + (size_t)(J.hist_off + ci) * kHistBins;
    const int64_t n = 2LL * J.F.W * J.F.H;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    uint8_t *fl = first_all + ((size_t)(smid % (uint32_t)nsm) * kChainWarps + warp) * kChainFirst + lane;
    uint32_t *tab = tab_all + warp * kChainTab;
    for (int i = threadIdx.x; i < (kHotBins + 32) / 4; i += kChainThreads) reinterpret_cast<uint4 *>(hot)[i] = make_uint4(0, 0, 0, 0);
    for (int i = lane; i < kChainTab / 4; i += 32) reinterpret_cast<uint4 *>(tab)[i] = make_uint4(~0u, ~0u, ~0u, ~0u);
    __syncthreads();
    // the lane's sub-range [lo, hi) of the warp's range
    const int sub = range_bytes >> 5;
    const int64_t ra = ((int64_t)seg * kChainWarps + warp) * range_bytes;
    const int64_t lo = min(n, ra + (int64_t)lane * sub), hi = min(n, lo + sub);
    const int len = (int)(hi - lo);
    const uint32_t slot = kHotBins + (uint32_t)lane;
    uint32_t *tl = tab + lane;
    if (len > 0) {
        uint32_t prev = S[lo == 0 ? n - 1 : lo - 1];  // cyclic predecessor
        const uint8_t *L = S + lo;                      // 16-byte aligned
        const int full = len >> 5;  // 32-byte steps, the next one loaded while this one is walked
        uint4 c0 = make_uint4(0, 0, 0, 0), c1 = c0;
        if (full > 0) {
            c0 = __ldg(reinterpret_cast<const uint4 *>(L));
            c1 = __ldg(reinterpret_cast<const uint4 *>(L) + 1);
        }
#pragma unroll 1
        for (int k = 0; k < full; k++) {
            uint4 n0 = make_uint4(0, 0, 0, 0), n1 = n0;
            if (k + 1 < full) {
                n0 = __ldg(reinterpret_cast<const uint4 *>(L + (size_t)(k + 1) * 32));
                n1 = __ldg(reinterpret_cast<const uint4 *>(L + (size_t)(k + 1) * 32) + 1);
            }
            const uint32_t w[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
            chain_walk32(w, prev, tl, fl, hot, ghist, slot);
            c0 = n0;
            c1 = n1;
        }
        for (int k = full << 5; k < len; k++) {  // ragged end of the stream
            const uint32_t b = L[k], a = prev;
            uint16_t *en = chain_entry(tl, b);
            const uint32_t e = *en;
            *en = (uint16_t)(a << kHotShift);
            if (e == kNoPred) fl[b * 32] = (uint8_t)a;
            chain_count(e, a, hot, ghist, slot);
            prev = b;
        }
    }
    __syncwarp();
    // stitch the lanes in order: a lane's first occurrence of b follows the
    // last occurrence in the nearest lower lane holding b. The warp's result
    // for b, (first << 16) | last (last as a table entry: p * 128, 0xFFFF:
    // none), then goes to word (b / 2) * 32 + b % 2 of its table, whose
    // entries are all read by then.
    // The first predecessors come from global memory 32 values ahead.
    const uint32_t lt = lanemask_lt();
    uint32_t keep = 0;
    uint32_t fv[32];
#pragma unroll
    for (int j = 0; j < 32; j++) fv[j] = __ldcg(fl + j * 32);
#pragma unroll 1
    for (int b0 = 0; b0 < 256; b0 += 32) {
        uint32_t fn[32];
#pragma unroll
        for (int j = 0; j < 32; j++) fn[j] = b0 + 32 < 256 ? __ldcg(fl + (b0 + 32 + j) * 32) : 0u;
#pragma unroll
        for (int j = 0; j < 32; j++) {
            const int b = b0 + j;
            const uint32_t last = *chain_entry(tl, b);
            const bool valid = last != kNoPred;
            const uint32_t m = __ballot_sync(LFC_FULL, valid);
            const uint32_t f = fv[j];  // meaningful where valid
            const uint32_t lower = m & lt;
            const uint32_t pl = __shfl_sync(LFC_FULL, last, lower ? 31 - __clz(lower) : lane);
            chain_count(valid && lower ? pl : kNoPred, f, hot, ghist, slot);
            const uint32_t f0 = __shfl_sync(LFC_FULL, f, m ? __ffs(m) - 1 : 0);
            const uint32_t lz = __shfl_sync(LFC_FULL, last, m ? 31 - __clz(m) : 0);
            const uint32_t res = (f0 << 16) | lz;
            if (j & 1) {
                __syncwarp();
                if (lane == 0) {
                    tab[(b >> 1) * 32] = keep;
                    tab[(b >> 1) * 32 + 1] = res;
                }
            } else {
                keep = res;
            }
        }
#pragma unroll
        for (int j = 0; j < 32; j++) fv[j] = fn[j];
    }
    __syncthreads();
    if (warp == 0) {  // the lanes' (0, 0) counts into bin (0, 0)
        const uint32_t z = warp_sum(hot[kHotBins + lane]);
        if (lane == 0 && z) hot[0] += z;
    }
    __syncthreads();
    constexpr int kFlush = 8;
    for (int i0 = threadIdx.x; i0 < kHot * kHot; i0 += kFlush * kChainThreads) {
        uint32_t v[kFlush];
#pragma unroll
        for (int j = 0; j < kFlush; j++) {
            const int i = i0 + j * kChainThreads;
            v[j] = i < kHot * kHot ? hot[i] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kFlush; j++) {
            const uint32_t i = (uint32_t)(i0 + j * kChainThreads), p = i / kHot, a = i % kHot;
            if (v[j]) atomicAdd(&ghist[(p << 8) | a], v[j]);
        }
    }
    // stitch the warps' ranges in order (thread per byte value)
    for (int bv = threadIdx.x; bv < 256; bv += kChainThreads) {
        uint32_t f0 = kNoPred, cur = kNoPred;
        for (int w = 0; w < kChainWarps; w++) {
            const uint32_t e = tab_all[w * kChainTab + (bv >> 1) * 32 + (bv & 1)];
            const uint32_t last = e & 0xFFFFu;  // p * 128
            if (last == kNoPred) continue;
            const uint32_t f = (e >> 16) & 255u;
            if (cur != kNoPred) atomicAdd(&ghist[(cur << (8 - kHotShift)) | f], 1u);  // (p << 8) | f
            else f0 = f;
            cur = last;
        }
        uint16_t *out = summ + (size_t)(J.summ_off + (int64_t)ci * J.segs + seg) * 512;
        out[bv] = (uint16_t)f0;
        out[256 + bv] = (uint16_t)(cur == kNoPred ? kNoPred : cur >> kHotShift);
    }
}

cudaError_t launch_emit_all(lfc_plan P, const JudgeFrame *d_frames, int nframes, const uint8_t *d_cand, int max_tiles,
                            int TS, int nslots_max, int any_temporal, int max_p) {
    const size_t smem = emit_all_smem_bytes(max_p, TS, nslots_max);
    bool planar = false;
    for (uint8_t id : P->ids_spatial) planar |= id_planar(id) != 0;
    for (uint8_t id : P->ids_temporal) planar |= id_planar(id) != 0;
    auto kern = planar ? emit_all_kernel<true> : emit_all_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(max_tiles, nframes, any_temporal ? 2 : 1);
    kern<<<grid, kEmitThreads, smem, P->stream>>>(d_frames, d_cand, P->ws.cstream, P->ws.cstream_slot,
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
        range_bytes, P->ws.chain_first, P->ws.chain_nsm);
    count_launches(P, 1);
    return cudaGetLastError();
}

}  // namespace lfc

// crc.cu -- CRC-32/BZIP2 (polynomial 0x04C11DB7, MSB first, init and final
// xor ~0) of byte ranges: the per-block CRC of the bzip2 format and the raw
// frame CRC of the container header.
//
// The register after a message M is I * x^(8|M|) + R(M) mod P, where R is
// the remainder with a zero register and is linear:
// R(A || B) = R(A) * x^(8|B|) + R(B). Chunks of a range are therefore
// reduced independently by table lookup, shifted by the bytes that follow
// them with a GF(2) multiply, and xor-ed together.
#include "lfc_common.cuh"

namespace lfc {

constexpr uint32_t kPoly = 0x04C11DB7u;
constexpr int kCrcChunk = 65536;  // bytes per partial remainder

__host__ __device__ constexpr uint32_t gf_mulmod(uint32_t a, uint32_t b) {
    uint32_t r = 0;
    for (int i = 31; i >= 0; i--) {
        r = (r & 0x80000000u) ? (r << 1) ^ kPoly : (r << 1);
        if ((b >> i) & 1u) r ^= a;
    }
    return r;
}

// x^(8k) mod P by square-and-multiply from x^8.
__host__ __device__ constexpr uint32_t x_pow_8k(uint64_t k) {
    uint32_t result = 1u, base = 0x100u;
    while (k) {
        if (k & 1) result = gf_mulmod(result, base);
        base = gf_mulmod(base, base);
        k >>= 1;
    }
    return result;
}

struct CrcChunk {
    const uint8_t *src;
    int32_t len;
    uint32_t shift;    // x^(8 * bytes of the range after this chunk) mod P
};

// T[k][i] = i * x^(32 + 8k) mod P: the effect of byte i followed by k zero
// bytes on a zero register, so four bytes fold in one step.
__device__ __forceinline__ void build_tables(uint32_t (*T)[256]) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        uint32_t v = (uint32_t)i << 24;
        for (int k = 0; k < 8; k++) v = (v & 0x80000000u) ? (v << 1) ^ kPoly : (v << 1);
        T[0][i] = v;
    }
    __syncthreads();
    for (int k = 1; k < 4; k++) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) {
            const uint32_t v = T[k - 1][i];
            T[k][i] = (v << 8) ^ T[0][v >> 24];
        }
        __syncthreads();
    }
}

// One CTA per chunk, seen as front-padded with zeros to kCrcChunk bytes
// (leading zeros leave a zero register unchanged): thread t reduces the
// 256-byte piece t four bytes at a time, then the warps merge their pieces
// in a shuffle tree (level j shifts the left half by x^(8 * 256 * 2^j)), the
// warps are merged in order, and the chunk remainder is shifted by the bytes
// of its range that follow it.
constexpr int kCrcPiece = kCrcChunk / 256;
// shuffle-tree level j merges halves of 2^j pieces; level 5 merges warps
__constant__ uint32_t c_crc_pow[6] = {x_pow_8k(kCrcPiece),      x_pow_8k(kCrcPiece * 2),  x_pow_8k(kCrcPiece * 4),
                                      x_pow_8k(kCrcPiece * 8),  x_pow_8k(kCrcPiece * 16), x_pow_8k(kCrcPiece * 32)};

__global__ void __launch_bounds__(256) crc_chunk_kernel(const CrcChunk *__restrict__ chunks, uint32_t *__restrict__ part) {
    __shared__ uint32_t T[4][256];
    __shared__ uint32_t red[8];
    build_tables(T);
    const CrcChunk c = chunks[blockIdx.x];
    const int pad = kCrcChunk - c.len;
    const int start = (int)threadIdx.x * kCrcPiece - pad;  // real offset of the piece
    uint32_t r = 0;
    if (start + kCrcPiece > 0) {
        const bool fast = start >= 0 && (((uintptr_t)(c.src + start)) & 3) == 0;
        for (int i = 0; i < kCrcPiece; i += 4) {
            uint32_t w;
            if (fast) {
                w = __byte_perm(__ldg(reinterpret_cast<const uint32_t *>(c.src + start + i)), 0u, 0x0123);
            } else {
                w = 0;
                for (int q = 0; q < 4; q++) {
                    const int o = start + i + q;
                    w = (w << 8) | (o >= 0 ? (uint32_t)c.src[o] : 0u);
                }
            }
            r ^= w;
            r = T[3][r >> 24] ^ T[2][(r >> 16) & 255u] ^ T[1][(r >> 8) & 255u] ^ T[0][r & 255u];
        }
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 5; j++) {
        const uint32_t rp = __shfl_xor_sync(LFC_FULL, r, 1 << j);
        const bool right = (lane >> j) & 1;
        r = gf_mulmod(right ? rp : r, c_crc_pow[j]) ^ (right ? r : rp);
    }
    if (lane == 0) red[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = red[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) t = gf_mulmod(t, c_crc_pow[5]) ^ red[i];
        part[blockIdx.x] = gf_mulmod(t, c.shift);
    }
}

// One thread per range: xor of its chunks' shifted remainders, plus the
// initial register shifted over the whole range (I * x^(8|M|)), complemented.
__global__ void crc_finish_kernel(const uint32_t *__restrict__ part, const int32_t *__restrict__ first_chunk,
                                  const uint32_t *__restrict__ init_shifted, int nranges, uint32_t *__restrict__ out,
                                  int out_stride_words) {
    const int rg = blockIdx.x * blockDim.x + threadIdx.x;
    if (rg >= nranges) return;
    uint32_t r = init_shifted[rg];
    for (int c = first_chunk[rg]; c < first_chunk[rg + 1]; c++) r ^= part[c];
    out[(size_t)rg * out_stride_words] = ~r;
}

// Descriptor tables of one CRC run, laid out in a caller-provided host
// buffer: [CrcChunk x nchunks] [int32 first_chunk x (n+1)] (pad 8)
// [uint32 I * x^(8 len) mod P x n]. Shifts are accumulated from each range's
// end, one GF(2) multiply per chunk.
int crc_count_chunks(const int64_t *len, int n) {
    int c = 0;
    for (int r = 0; r < n; r++) c += (int)((len[r] + kCrcChunk - 1) / kCrcChunk);
    return c;
}

size_t crc_table_bytes(int nchunks, int n) {
    size_t o = (size_t)nchunks * sizeof(CrcChunk) + (size_t)(n + 1) * 4;
    o = (o + 7) & ~(size_t)7;
    return o + (size_t)n * 8;
}

void crc_build_tables(const uint8_t *const *ptr, const int64_t *len, int n, uint8_t *out, CrcRun *run) {
    constexpr uint32_t kFullShift = x_pow_8k(kCrcChunk);
    CrcChunk *ch = reinterpret_cast<CrcChunk *>(out);
    int k = 0;
    std::vector<int32_t> first(n + 1);
    std::vector<uint32_t> init(n);
    for (int r = 0; r < n; r++) {
        first[r] = k;
        const int nc = (int)((len[r] + kCrcChunk - 1) / kCrcChunk);
        uint32_t acc = 1u;  // x^(8 * bytes after the chunk)
        for (int i = nc - 1; i >= 0; i--) {
            const int64_t o = (int64_t)i * kCrcChunk;
            CrcChunk c;
            c.src = ptr[r] + o;
            c.len = (int32_t)(len[r] - o < kCrcChunk ? len[r] - o : kCrcChunk);
            c.shift = acc;
            memcpy(&ch[k + i], &c, sizeof(c));
            acc = gf_mulmod(acc, c.len == kCrcChunk ? kFullShift : x_pow_8k((uint64_t)c.len));
        }
        init[r] = gf_mulmod(0xFFFFFFFFu, acc);
        k += nc;
    }
    first[n] = k;
    size_t o = (size_t)k * sizeof(CrcChunk);
    memcpy(out + o, first.data(), (size_t)(n + 1) * 4);
    run->off_first = o;
    o += (size_t)(n + 1) * 4;
    o = (o + 7) & ~(size_t)7;
    memcpy(out + o, init.data(), (size_t)n * 4);
    run->off_len = o;
    run->nchunks = k;
    run->nranges = n;
}

// Launches a CRC run whose tables sit at d_tables (device).
cudaError_t launch_crc(lfc_plan P, const uint8_t *d_tables, const CrcRun &run, uint32_t *out, int out_stride_words,
                       cudaStream_t stream, uint32_t *part) {
    if (run.nchunks > P->ws.crc_part_cap) return cudaErrorInvalidValue;
    if (!stream) stream = P->stream;
    if (!part) part = P->ws.crc_part;
    if (run.nchunks) crc_chunk_kernel<<<(unsigned)run.nchunks, 256, 0, stream>>>(reinterpret_cast<const CrcChunk *>(d_tables), part);
    crc_finish_kernel<<<(run.nranges + 127) / 128, 128, 0, stream>>>(
        part, reinterpret_cast<const int32_t *>(d_tables + run.off_first),
        reinterpret_cast<const uint32_t *>(d_tables + run.off_len), run.nranges, out, out_stride_words);
    count_launches(P, run.nchunks ? 2 : 1);
    return cudaGetLastError();
}

// Immediate form: stage the tables in the plan's descriptor buffer first.
static cudaError_t run_ranges(lfc_plan P, const uint8_t *const *ptr, const int64_t *len, int n, uint32_t *out,
                              int out_stride_words) {
    const int nchunks = crc_count_chunks(len, n);
    std::vector<uint8_t> blob(crc_table_bytes(nchunks, n));
    CrcRun run;
    crc_build_tables(ptr, len, n, blob.data(), &run);
    if (blob.size() > P->ws.chunk_desc_bytes) return cudaErrorInvalidValue;
    uint8_t *d = reinterpret_cast<uint8_t *>(P->ws.chunk_desc);
    cudaError_t e = cudaMemcpyAsync(d, blob.data(), blob.size(), cudaMemcpyHostToDevice, P->stream);
    if (e != cudaSuccess) return e;  // pageable source: staged before the call returns
    return launch_crc(P, d, run, out, out_stride_words);
}

cudaError_t launch_block_crc(lfc_plan P, const BlockDesc *h_blocks, int nblocks, BlockState *d_state) {
    std::vector<const uint8_t *> ptr(nblocks);
    std::vector<int64_t> len(nblocks);
    for (int b = 0; b < nblocks; b++) { ptr[b] = h_blocks[b].src; len[b] = h_blocks[b].len; }
    static_assert(sizeof(BlockState) % 4 == 0, "BlockState words");
    return run_ranges(P, ptr.data(), len.data(), nblocks, &d_state[0].crc, (int)(sizeof(BlockState) / 4));
}

cudaError_t launch_range_crc(lfc_plan P, const uint8_t *const *h_ptr, const int64_t *h_len, int n, uint32_t *d_out) {
    return run_ranges(P, h_ptr, h_len, n, d_out, 1);
}

}  // namespace lfc

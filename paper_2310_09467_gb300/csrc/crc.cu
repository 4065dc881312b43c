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

__device__ __forceinline__ uint32_t gf_mulmod(uint32_t a, uint32_t b) {
    uint32_t r = 0;
#pragma unroll 8
    for (int i = 31; i >= 0; i--) {
        r = (r & 0x80000000u) ? (r << 1) ^ kPoly : (r << 1);
        if ((b >> i) & 1u) r ^= a;
    }
    return r;
}

// x^(8k) mod P by square-and-multiply from x^8.
__device__ __forceinline__ uint32_t x_pow_8k(uint64_t k) {
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
    int32_t range;     // which range this chunk belongs to
    int64_t after;     // bytes of the range after this chunk
};

__device__ __forceinline__ void build_table(uint32_t *tab) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        uint32_t v = (uint32_t)i << 24;
        for (int k = 0; k < 8; k++) v = (v & 0x80000000u) ? (v << 1) ^ kPoly : (v << 1);
        tab[i] = v;
    }
}

// One CTA per chunk: each thread reduces a contiguous piece, then the pieces
// are shifted into place and xor-reduced; the chunk's remainder is shifted
// by the bytes of its range that follow it.
__global__ void __launch_bounds__(256) crc_chunk_kernel(const CrcChunk *__restrict__ chunks, uint32_t *__restrict__ part) {
    __shared__ uint32_t tab[256];
    __shared__ uint32_t red[8];
    build_table(tab);
    __syncthreads();
    const CrcChunk c = chunks[blockIdx.x];
    const int per = (c.len + blockDim.x - 1) / blockDim.x;
    const int a = min(c.len, (int)threadIdx.x * per), e = min(c.len, a + per);
    uint32_t r = 0;
    for (int i = a; i < e; i++) r = (r << 8) ^ tab[(r >> 24) ^ c.src[i]];
    if (e > a) r = gf_mulmod(r, x_pow_8k((uint64_t)(c.len - e) + (uint64_t)c.after));
    for (int o = 16; o > 0; o >>= 1) r ^= __shfl_xor_sync(LFC_FULL, r, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t ^= red[i];
        part[blockIdx.x] = t;
    }
}

// One thread per range: xor of its chunks' shifted remainders, plus the
// shifted initial register, complemented.
__global__ void crc_finish_kernel(const uint32_t *__restrict__ part, const int32_t *__restrict__ first_chunk,
                                  const int64_t *__restrict__ range_len, int nranges, uint32_t *__restrict__ out,
                                  int out_stride_words) {
    const int rg = blockIdx.x * blockDim.x + threadIdx.x;
    if (rg >= nranges) return;
    uint32_t r = 0;
    for (int c = first_chunk[rg]; c < first_chunk[rg + 1]; c++) r ^= part[c];
    r ^= gf_mulmod(0xFFFFFFFFu, x_pow_8k((uint64_t)range_len[rg]));
    out[(size_t)rg * out_stride_words] = ~r;
}

// Descriptor tables of one CRC run, laid out in a caller-provided host
// buffer: [CrcChunk x nchunks] [int32 first_chunk x (n+1)] (pad 8)
// [int64 range_len x n].
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
    CrcChunk *ch = reinterpret_cast<CrcChunk *>(out);
    int k = 0;
    std::vector<int32_t> first(n + 1);
    for (int r = 0; r < n; r++) {
        first[r] = k;
        for (int64_t o = 0; o < len[r]; o += kCrcChunk) {
            CrcChunk c;
            c.src = ptr[r] + o;
            c.len = (int32_t)(len[r] - o < kCrcChunk ? len[r] - o : kCrcChunk);
            c.range = r;
            c.after = len[r] - o - c.len;
            memcpy(&ch[k++], &c, sizeof(c));
        }
    }
    first[n] = k;
    size_t o = (size_t)k * sizeof(CrcChunk);
    memcpy(out + o, first.data(), (size_t)(n + 1) * 4);
    run->off_first = o;
    o += (size_t)(n + 1) * 4;
    o = (o + 7) & ~(size_t)7;
    memcpy(out + o, len, (size_t)n * 8);
    run->off_len = o;
    run->nchunks = k;
    run->nranges = n;
}

// Launches a CRC run whose tables sit at d_tables (device).
cudaError_t launch_crc(lfc_plan P, const uint8_t *d_tables, const CrcRun &run, uint32_t *out, int out_stride_words) {
    if (run.nchunks > P->ws.crc_part_cap) return cudaErrorInvalidValue;
    if (run.nchunks) crc_chunk_kernel<<<(unsigned)run.nchunks, 256, 0, P->stream>>>(reinterpret_cast<const CrcChunk *>(d_tables), P->ws.crc_part);
    crc_finish_kernel<<<(run.nranges + 127) / 128, 128, 0, P->stream>>>(
        P->ws.crc_part, reinterpret_cast<const int32_t *>(d_tables + run.off_first),
        reinterpret_cast<const int64_t *>(d_tables + run.off_len), run.nranges, out, out_stride_words);
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

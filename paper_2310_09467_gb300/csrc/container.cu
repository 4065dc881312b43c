// container.cu -- the compressed file of one frame (Sec. 2.1.4: header with
// the 8-bit predictor id; Sec. 2.1.3: block information, then the blocks'
// coded data in order). Little-endian header:
//   0 "LFC1" | 4 u16 version 1 | 6 u16 flags (bit 0 temporal) | 8 u32 W |
//   12 u32 H | 16 u32 pitch | 20 u8 id + 3 zero bytes | 24 u32 block_bytes |
//   28 u32 n_blocks | 32 u32 raw-frame CRC | 36 u32 header bytes |
//   40 u32 stream bytes per block | streams.
#include "lfc_common.cuh"

namespace lfc {

__device__ __forceinline__ void st32(uint8_t *p, uint32_t v) {
    p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}

// One warp per frame: header, block table, destination of every stream.
__global__ void container_header_kernel(const FrameOut *__restrict__ fo, int nframes, const BlockState *__restrict__ st,
                                        const uint8_t *__restrict__ choice, const uint32_t *__restrict__ frame_crc,
                                        uint8_t *__restrict__ out, uint64_t *__restrict__ out_sizes,
                                        uint64_t *__restrict__ block_dst, int block_bytes) {
    const int f = blockIdx.x;
    if (f >= nframes) return;
    const FrameOut F = fo[f];
    uint8_t *o = out + F.out_off;
    const uint32_t hdr = 40u + 4u * (uint32_t)F.nblocks;
    if (threadIdx.x == 0) {
        const int id = choice[f];
        o[0] = 'L'; o[1] = 'F'; o[2] = 'C'; o[3] = '1';
        o[4] = 1; o[5] = 0;
        o[6] = (uint8_t)((id >> 7) & 1); o[7] = 0;
        st32(o + 8, (uint32_t)F.W);
        st32(o + 12, (uint32_t)F.H);
        st32(o + 16, (uint32_t)F.p);
        o[20] = (uint8_t)id; o[21] = 0; o[22] = 0; o[23] = 0;
        st32(o + 24, (uint32_t)block_bytes);
        st32(o + 28, (uint32_t)F.nblocks);
        st32(o + 32, frame_crc[f]);
        st32(o + 36, hdr);
        uint64_t pos = hdr;
        for (int k = 0; k < F.nblocks; k++) {
            const uint32_t sb = st[F.block0 + k].stream_bytes;
            st32(o + 40 + 4 * k, sb);
            block_dst[F.block0 + k] = F.out_off + pos;
            pos += sb;
        }
        out_sizes[f] = pos;
    }
}

// Grid (chunk, block): copy stream bytes to their destinations.
__global__ void copy_streams_kernel(const BlockState *__restrict__ st, const uint32_t *__restrict__ packed_all,
                                    int64_t stream_words, const uint64_t *__restrict__ block_dst, uint8_t *__restrict__ out,
                                    size_t stride, uint32_t *__restrict__ sizes) {
    const int b = blockIdx.y;
    const uint32_t nbytes = st[b].stream_bytes;
    const uint8_t *src = reinterpret_cast<const uint8_t *>(packed_all + (size_t)b * stream_words);
    uint8_t *dst = block_dst ? out + block_dst[b] : out + (size_t)b * stride;
    if (sizes && blockIdx.x == 0 && threadIdx.x == 0) sizes[b] = nbytes;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nbytes; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

cudaError_t launch_container(lfc_plan P, int nframes, int nblocks, const FrameOut *d_fo, const uint8_t *d_choice,
                             const uint32_t *d_frame_crc, uint8_t *d_out, uint64_t *d_out_sizes, int block_bytes) {
    Workspace &ws = P->ws;
    container_header_kernel<<<nframes, 32, 0, P->stream>>>(d_fo, nframes, ws.bstate, d_choice, d_frame_crc, d_out,
                                                           d_out_sizes, ws.block_dst, block_bytes);
    dim3 grid(64, nblocks);
    copy_streams_kernel<<<grid, 256, 0, P->stream>>>(ws.bstate, ws.packed, ws.stream_words, ws.block_dst, d_out, 0, nullptr);
    count_launches(P, 2);
    return cudaGetLastError();
}

cudaError_t launch_copy_streams(lfc_plan P, int nblocks, uint8_t *d_out, size_t stride, uint32_t *d_sizes) {
    Workspace &ws = P->ws;
    dim3 grid(64, nblocks);
    copy_streams_kernel<<<grid, 256, 0, P->stream>>>(ws.bstate, ws.packed, ws.stream_words, nullptr, d_out, stride, d_sizes);
    count_launches(P, 1);
    return cudaGetLastError();
}

}  // namespace lfc

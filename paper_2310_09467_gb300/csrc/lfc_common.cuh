// lfc_common.cuh -- internal declarations shared by the liblfc CUDA sources.
// Nothing here is part of the public ABI (include/lfc.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <cstring>
#include <string>
#include <vector>

#include "lfc.h"

namespace lfc {

// ---------------------------------------------------------------- constants
constexpr int kMaxBlockBytes = LFC_MAX_BLOCK_BYTES;  // input bytes per bzip2 block
constexpr int kTile = 4096;                          // elements per sort tile
constexpr int kRleCap = 900000;                      // RLE1 output bound (5/4 of 720000)
constexpr int kBlockCap = 901120;                    // 220 tiles of 4096, >= kRleCap
constexpr int kTilesPerBlock = kBlockCap / kTile;    // 220
constexpr int kMaxAlpha = 258;                       // bzip2 symbols: 256 MTF + RUNA/RUNB... + EOB
constexpr int kMaxGroups = 6;
constexpr int kMaxSelectors = 18002;
constexpr int kHistBins = 65536;
constexpr int kMaxCand = 104;                        // candidates per frame: 26 default ids x 2 byte layouts x 2 (temporal)
constexpr int kSortCtlHead = 16;                     // sort state words before the per-block tile offsets
constexpr int kSortFaultWord = 5;                    // sort state word of the fault-injection test hook
constexpr int kSortStickyWord = 9;                   // sort state word kept until lfc_plan_device_status reads it

#define LFC_FULL 0xffffffffu

// ------------------------------------------------------------ warp helpers
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << lane_id()) - 1u; }
__device__ __forceinline__ uint32_t lanemask_gt() { return lane_id() == 31 ? 0u : (~0u << (lane_id() + 1)); }

template <typename T>
__device__ __forceinline__ T warp_incl_sum(T v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(LFC_FULL, v, o);
        if ((int)lane_id() >= o) v += t;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(LFC_FULL, v, o);
    return v;
}

__device__ __forceinline__ int warp_incl_max(int v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(LFC_FULL, v, o);
        if ((int)lane_id() >= o) v = max(v, t);
    }
    return v;
}

// Block-wide exclusive sum over blockDim.x threads (<= 1024). `sh` needs 33
// entries. Returns the exclusive prefix; *total gets the block sum.
template <typename T>
__device__ __forceinline__ T block_excl_sum(T v, T *sh, T *total) {
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    T incl = warp_incl_sum(v);
    if (lane_id() == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        T s = lane_id() < (uint32_t)nw ? sh[lane_id()] : T(0);
        T si = warp_incl_sum(s);
        if (lane_id() < (uint32_t)nw) sh[lane_id()] = si - s;
        if (lane_id() == 31) sh[32] = si;
    }
    __syncthreads();
    T r = sh[w] + incl - v;
    if (total) *total = sh[32];
    __syncthreads();
    return r;
}

// Block-wide exclusive max over blockDim.x threads (identity -1).
__device__ __forceinline__ int block_excl_max(int v, int *sh) {
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int incl = warp_incl_max(v);
    if (lane_id() == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        int s = lane_id() < (uint32_t)nw ? sh[lane_id()] : -1;
        int si = warp_incl_max(s);
        int ex = __shfl_up_sync(LFC_FULL, si, 1);
        if (lane_id() == 0) ex = -1;
        if (lane_id() < (uint32_t)nw) sh[lane_id()] = ex;
    }
    __syncthreads();
    int ex_in_warp = __shfl_up_sync(LFC_FULL, incl, 1);
    if (lane_id() == 0) ex_in_warp = -1;
    int r = max(sh[w], ex_in_warp);
    __syncthreads();
    return r;
}

// ------------------------------------------------------------ candidate ids
// Fields of a candidate id (include/lfc.h): f bits 0-2, byte layout bit 3
// (1: planar, high bytes then low bytes), domain bits 4-5, ordering bit 6,
// temporal bit 7.
__host__ __device__ __forceinline__ int id_f(int id) { return id & 7; }
__host__ __device__ __forceinline__ int id_planar(int id) { return (id >> 3) & 1; }
__host__ __device__ __forceinline__ int id_dom(int id) { return (id >> 4) & 3; }
__host__ __device__ __forceinline__ int id_ord(int id) { return (id >> 6) & 1; }
__host__ __device__ __forceinline__ int id_tmp(int id) { return (id >> 7) & 1; }

// ------------------------------------------------------------- descriptors
// One frame as the kernels see it.
struct FrameDev {
    const uint16_t *X;     // raw counts, row-major H x W
    const uint16_t *prev;  // previous raw frame or nullptr
    int32_t W, H, p, Nx, Ny;
};

// Judge work description of one frame.
struct JudgeFrame {
    FrameDev F;
    int32_t K;             // candidates judged
    int32_t cand_off;      // first entry in the candidate id table
    int32_t segs;          // segments (CTAs) per candidate
    int32_t rows_per_seg;  // stream rows per segment
    int64_t cta_base;      // first CTA index of this frame
    int64_t hist_off;      // first histogram (in units of 65536 bins)
    int64_t summ_off;      // first segment summary
    const uint64_t *mask;  // candidate mask (4 words) from the proposal, or nullptr = all
};

__device__ __forceinline__ bool cand_on(const JudgeFrame &J, int id) {
    return J.mask == nullptr || ((J.mask[id >> 6] >> (id & 63)) & 1ull);
}

// One bzip2 block: input bytes at src[0 .. len).
struct BlockDesc {
    const uint8_t *src;
    int32_t len;
    int32_t frame;         // owning frame (-1 for raw block encodes)
};

// Per-block coder state on the device (sizes the host never reads).
struct BlockState {
    int32_t m;             // RLE1 output length
    int32_t orig_ptr;      // BWT origin row
    int32_t n_act;         // active elements in the current doubling round
    int32_t n_act_next;    // active elements after the round
    int32_t n_mtf;         // bzip2 symbols including EOB
    int32_t n_in_use;      // distinct bytes in the block
    int32_t n_groups;
    int32_t n_sel;
    uint32_t crc;          // CRC-32/BZIP2 of the block input (word 8)
    uint32_t stream_bytes; // packed stream length
    uint32_t stream_bits;
    uint32_t data_bit0;    // first bit of the Huffman-coded data in the stream
    uint32_t in_use[8];    // bytes present in the block
};
static_assert(sizeof(BlockState) == 80, "BlockState layout");

// ------------------------------------------------------------------ plan
struct Workspace {
    // judge
    uint32_t *hist = nullptr;      // judge_frames_cap * K * 65536
    uint16_t *summ = nullptr;      // per judge CTA: first[256], last[256]
    uint8_t *chain_first = nullptr;  // per SM: the chain kernel's first-predecessor bytes
    int chain_nsm = 0;               // SM slots of chain_first (%nsmid)
    uint64_t *scores = nullptr;    // max_frames * 256
    uint8_t *choice = nullptr;     // max_frames
    JudgeFrame *jframes = nullptr; // judge_frames_cap
    uint8_t *cand = nullptr;       // judge_frames_cap * kMaxCand
    uint64_t *l2tab = nullptr;     // 65536
    int64_t summ_cap = 0;
    uint8_t *cstream = nullptr;    // candidate streams: judge_frames_cap * cstream_kmax slots
    // lfc_compress_host staging, allocated on its first call: frames, previous
    // frames, containers, sizes, given ids
    uint8_t *hx_frames = nullptr, *hx_prev = nullptr, *hx_out = nullptr, *hx_choice = nullptr;
    uint64_t *hx_sizes = nullptr;
    size_t hx_out_cap = 0;
    uint64_t *masks = nullptr;     // proposal candidate masks, max_frames x 4
    uint8_t *class_ids = nullptr;  // proposal class -> candidate id (64)
    int64_t cstream_slot = 0;
    int cstream_kmax = 0;
    // symbol streams of the frames being compressed
    uint8_t *stream = nullptr;     // max_frames * stream_slot
    int64_t stream_slot = 0;
    // coder, per block slot
    BlockDesc *blocks = nullptr;
    BlockState *bstate = nullptr;
    uint8_t *rle = nullptr;        // block_cap * kBlockCap
    int32_t *sa = nullptr;         // block_cap * kBlockCap
    int32_t *sa2 = nullptr;
    int32_t *rank = nullptr;
    int32_t *act = nullptr;        // active SA positions
    int32_t *act2 = nullptr;
    int32_t *val = nullptr;        // SA values of the active elements
    int32_t *val2 = nullptr;
    uint64_t *keys = nullptr;      // sort keys riding with sa / val, block_cap * kBlockCap
    uint64_t *keys2 = nullptr;
    uint32_t *lbstat = nullptr;    // radix look-back status, 2 arrays of block_cap * kTilesPerBlock * 256
    size_t lbstat_words = 0;       // words of one of those arrays
    uint32_t *dhist = nullptr;     // per block and radix pass: digit totals, block_cap * 8 * 256
    int32_t *segbig = nullptr;     // per block: a doubling round has a group longer than the segmented sort's window
    int32_t *tileaux = nullptr;    // block_cap * kTilesPerBlock * 4
    uint8_t *bwt = nullptr;        // L column
    uint8_t *mtfidx = nullptr;
    uint8_t *mtflists = nullptr;   // block_cap * kTilesPerBlock * 256
    uint8_t *mtfrec = nullptr;     // recency lists, same shape
    int32_t *mtfreclen = nullptr;  // block_cap * kTilesPerBlock
    uint16_t *sym = nullptr;       // block_cap * (kBlockCap + 1)
    uint32_t *freq = nullptr;      // block_cap * kMaxAlpha
    uint32_t *rfreq = nullptr;     // block_cap * kMaxGroups * kMaxAlpha, counts of a refinement pass
    uint8_t *sel = nullptr;        // block_cap * kMaxSelectors
    uint8_t *lens = nullptr;       // block_cap * 6 * 258
    uint32_t *codes = nullptr;     // block_cap * 6 * 258
    uint32_t *packed = nullptr;    // block_cap * stream_words
    int64_t stream_words = 0;
    int32_t *act_total = nullptr;  // sort state: kSortCtlHead words + block_cap + 1 tile offsets
    int32_t *h_act_total = nullptr;// pinned host mirror of the first kSortCtlHead words
    // container assembly
    uint64_t *block_dst = nullptr;     // block_cap: stream destination offsets
    uint32_t *frame_crc = nullptr;     // max_frames
    uint32_t *crc_part = nullptr;      // CRC partial remainders
    uint32_t *crc_part2 = nullptr;   // partial remainders of the frame CRCs (side stream)
    int64_t crc_part_cap = 0;
    void *chunk_desc = nullptr;        // descriptor staging (CRC chunks, frame tables)
    size_t chunk_desc_bytes = 0;
    // decode
    uint8_t *dec_tt = nullptr;
};

}  // namespace lfc

struct lfc_plan_s {
    lfc_config cfg;
    cudaStream_t stream = nullptr;
    cudaStream_t aux_stream = nullptr;  // capture of conditional-node bodies
    cudaStream_t side_stream = nullptr; // CRCs, overlapped with the judge and the BWT
    cudaEvent_t side_fork = nullptr, side_join = nullptr;
    cudaStream_t cap_stream = nullptr;  // capture of batches
    int device = 0;
    int sm_count = 0;  // streaming multiprocessors of the device
    std::string err;
    std::vector<uint8_t> ids_spatial;   // judged for every frame
    std::vector<uint8_t> ids_temporal;  // judged for frames with prev
    int judge_frames_cap = 0;           // frames per judge launch (allocated)
    lfc_tuning tune{16, 262144, 0, 0};    // autotuned judge knobs
    lfc_cnn cnn = nullptr;              // learned proposal (optional)
    int topk = 0;
    float tau = 0.f;
    int block_cap = 0;                  // blocks per coder pass
    lfc::Workspace ws;
    // tracing: CUDA events around stages, harvested by lfc_plan_timing
    bool timing = false;
    int64_t launches = 0;
    struct Span { int stage; cudaEvent_t a, b; };
    std::vector<Span> spans;
    std::vector<cudaEvent_t> event_pool;
    cudaEvent_t open_ev[LFC_NUM_STAGES] = {};
    double stage_ms[LFC_NUM_STAGES] = {};
    int64_t bwt_calls = 0, bwt_rounds = 0, bwt_tied_total = 0, bwt_elements = 0, bwt_elements_in = 0;
    int64_t bwt_round_tied[32] = {};
    long long wait_cycles = 0;          // bounded device waits: budget in SM clock cycles
    int sm_clock_khz = 0;
    bool bwt_timed_out = false;         // a wait of the last suffix sort gave up
    int64_t stage_spans[LFC_NUM_STAGES] = {};
};

namespace lfc {

// cnn.cu
int cnn_propose(lfc_cnn C, const lfc_frame *frames, int n, const uint8_t *d_class_ids, int topk, float tau,
                uint64_t *d_masks, cudaStream_t s);
int cnn_classes(lfc_cnn C);
int cnn_max_batch(lfc_cnn C);

// ---------------------------------------------------------------- tracing
void stage_begin(lfc_plan P, int stage);
void stage_end(lfc_plan P, int stage);
inline void count_launches(lfc_plan P, int n) { P->launches += n; }

// ------------------------------------------------------- internal launchers
// judge.cu
cudaError_t init_l2_table(uint64_t *tab, cudaStream_t s);
size_t judge_smem_bytes(int maxW);
// judge_stream.cu
size_t emit_all_smem_bytes(int p, int ts, int nslots);
size_t chain_smem_bytes();
int64_t chain_seg_bytes(int range_bytes);  // stream bytes one chain CTA covers
size_t chain_first_bytes(int nsm);          // chain_first bytes for nsm SM slots
cudaError_t query_nsmid(cudaStream_t s, int *nsm);
cudaError_t launch_emit_all(lfc_plan P, const JudgeFrame *d_frames, int nframes, const uint8_t *d_cand, int max_tiles,
                            int TS, int nslots_max, int any_temporal, int max_p);
cudaError_t launch_chain_hist(lfc_plan P, const JudgeFrame *d_frames, int nframes, const uint8_t *d_cand, int64_t total_ctas,
                              int range_bytes);
struct JudgeLaunch {
    int max_tiles, TS, nslots_max, any_temporal, max_p, range_bytes;
};
cudaError_t launch_judge(lfc_plan P, const JudgeFrame *d_frames, int nframes, int64_t total_ctas,
                         const JudgeLaunch &L, const uint8_t *d_cand, int64_t nhist,
                         uint64_t *d_scores, uint8_t *d_choice);
cudaError_t launch_copy_chosen(lfc_plan P, const JudgeFrame *d_frames, int nframes, const uint8_t *d_cand,
                               const uint8_t *d_choice, uint8_t *const *d_dst);
cudaError_t launch_emit(const FrameDev *h_frames, const uint8_t *d_choice, int nframes,
                        uint8_t *const *h_dst, cudaStream_t s);
cudaError_t launch_symbols_one(const FrameDev &F, int id, uint16_t *dst, cudaStream_t s);

// crc.cu
struct CrcRun {
    int nchunks = 0, nranges = 0;
    size_t off_first = 0, off_len = 0;
};
int crc_count_chunks(const int64_t *len, int n);
size_t crc_table_bytes(int nchunks, int n);
void crc_build_tables(const uint8_t *const *ptr, const int64_t *len, int n, uint8_t *out, CrcRun *run);
cudaError_t launch_crc(lfc_plan P, const uint8_t *d_tables, const CrcRun &run, uint32_t *out, int out_stride_words,
                       cudaStream_t stream = nullptr, uint32_t *part = nullptr);
cudaError_t launch_block_crc(lfc_plan P, const BlockDesc *h_blocks, int nblocks, BlockState *d_state);
cudaError_t launch_range_crc(lfc_plan P, const uint8_t *const *h_ptr, const int64_t *h_len, int n,
                             uint32_t *d_out);

// bwt.cu
cudaError_t launch_rle1(lfc_plan P, int nblocks, const BlockDesc *d_blocks);
cudaError_t launch_bwt(lfc_plan P, int nblocks, int max_m);
cudaError_t launch_copy_bwt(lfc_plan P, int nblocks, uint8_t *d_L, size_t stride, uint32_t *d_len, uint32_t *d_orig);

// mtf_huff.cu
cudaError_t launch_mtf_rle2(lfc_plan P, int nblocks);
cudaError_t launch_huffman(lfc_plan P, int nblocks);
cudaError_t launch_pack(lfc_plan P, int nblocks);

// container.cu
struct FrameOut {
    uint64_t out_off;    // container offset in d_out
    int32_t block0, nblocks;
    int32_t W, H, p, pad;
};
cudaError_t launch_container(lfc_plan P, int nframes, int nblocks, const FrameOut *d_fo, const uint8_t *d_choice,
                             const uint32_t *d_frame_crc, uint8_t *d_out, uint64_t *d_out_sizes, int block_bytes);
cudaError_t launch_copy_streams(lfc_plan P, int nblocks, uint8_t *d_out, size_t stride, uint32_t *d_sizes);

// decode.cu
struct DecBlockHost {
    const uint8_t *src;
    int64_t src_len;
    uint8_t *dst;
    int32_t expect;
    int32_t pad;
};
cudaError_t launch_bzip2_decode(lfc_plan P, const void *d_blocks, int nblocks, int32_t *d_status);
cudaError_t launch_inverse_predict(lfc_plan P, const uint16_t *Z, const uint16_t *prev, uint16_t *X, int32_t *E,
                                   int W, int H, int p, int id);

}  // namespace lfc

/*
 * lfc.h -- C ABI of liblfc, a GB300 (sm_103a) implementation of the PC-bzip2
 * compression path for raw light-field microscopy frames (Su et al.,
 * "PC-bzip2: a phase-space continuity enhanced lossless compression
 * algorithm for light field microscopy data").
 *
 * Pipeline (Fig. 1c and Fig. 2 of the paper): predict every candidate
 * (Sec. 2.1.1), score each by the two-dimensional image entropy of Eq. (1)
 * (Sec. 2.1.2), keep the best, bzip2-code the chosen stream in independent
 * blocks (Sec. 2.1.3) and pack a header holding the 8-bit predictor id
 * (Sec. 2.1.4). Every stage runs in this library's CUDA kernels.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are device pointers, h_* are host pointers.
 *  - The caller owns every input and output buffer. A plan owns its
 *    workspace, allocated once by lfc_plan_create; no other call allocates
 *    device memory.
 *  - Calls are asynchronous on the plan's stream unless they say otherwise;
 *    results are ready once that stream is synchronised.
 *  - The return value is an lfc_status. On LFC_ERR_* nothing is guaranteed
 *    about outputs. lfc_plan_last_error gives a one-line reason.
 *  - All integers in formats are little-endian. The arithmetic is integer
 *    throughout and bit-exact; no call has a CPU fallback.
 */
#ifndef LFC_H
#define LFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LFC_OK = 0,
    LFC_ERR_INVALID_ARG = 1,   /* argument outside its documented range */
    LFC_ERR_CAPACITY = 2,      /* an output buffer is smaller than required */
    LFC_ERR_CORRUPT = 3,       /* a container or bzip2 stream failed a check */
    LFC_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    LFC_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    LFC_ERR_UNIMPLEMENTED = 6, /* feature not built */
    LFC_ERR_NOMEM = 7          /* workspace allocation failed at plan creation */
} lfc_status;

/* Candidate (predictor) id: one unsigned 8-bit integer, stored in the header
 * (Sec. 2.1.4). The paper's mapping table (Fig. 3) is not available; this
 * library's layout is
 *   bits 0-2  f: 0 none, 1 A, 2 B, 3 C, 4 A+B-C, 5 A+(B-C)/2, 6 B+(A-C)/2,
 *             7 (A+B)/2  -- the lossless-JPEG set of Sec. 3 / Fig. 3b, with
 *             A = left, B = top, C = top-left and floor division;
 *   bit  3    byte layout of the realigned stream (Sec. 2.1.2, Fig. 2c):
 *             0 (lo, hi) per symbol, 1 planar -- the high bytes of all
 *             symbols in stream order, then their low bytes;
 *   bits 4-5  domain: 0 intra-lenslet (neighbouring pixels in one microlens),
 *             1 inter-lenslet (same pixel of the neighbouring microlenses),
 *             2 phase space (intra residual predicted again across
 *             microlenses) -- Sec. 2.1.1, Fig. 1b, Fig. 3c;
 *   bit  6    ordering: 0 raw lenslet-major layout, 1 view-major mosaic
 *             out[v*Ny + t][u*Nx + s] = in[t*p + v][s*p + u];
 *   bit  7    temporal: predict the difference to the previous raw frame.
 * Valid ids: domain <= 2, and f == 0 only with domain 0. */
#define LFC_ID(f, domain, ordering, temporal) \
    ((uint8_t)((f) | ((domain) << 4) | ((ordering) << 6) | ((temporal) << 7)))
#define LFC_ID_PLANAR(id) ((uint8_t)((id) | 8))

/* Largest input block per bzip2 stream. RLE1 grows a block by at most 5/4,
 * so a block always fits one level-9 bzip2 block (900000 bytes). */
#define LFC_MAX_BLOCK_BYTES 720000

typedef struct lfc_plan_s *lfc_plan;

typedef struct {
    /* Largest frame the plan serves (workspace sizing). width and height
     * must be multiples of pitch; 2 * width * height <= 2^26. */
    int32_t width, height, pitch;
    /* Most frames one call may pass. */
    int32_t max_frames;
    /* Candidate set, one bit per id (bit id % 64 of word id / 64). All zero
     * selects the default set: f in {0, 4, 5, 6, 7} x 3 domains (f = 0 only
     * in domain 0) x 2 orderings = 26 ids, plus the same 26 with the temporal
     * bit for frames that carry a previous frame. Temporal ids in the mask
     * apply only to frames with prev != NULL. */
    uint64_t candidate_mask[4];
    /* Nonzero enables temporal candidates for frames that pass prev. */
    int32_t temporal;
    /* Informational for callers building series (keyframe every G frames:
     * pass prev = NULL on keyframes). Default 16. */
    int32_t keyframe_interval;
    /* Input bytes per bzip2 block; 0 selects 720000. 1 .. 720000. */
    int32_t block_bytes;
    /* Learned proposal: judge only the top-k ids of the proposal network,
     * all ids if its top probability is below tau. 0 = exhaustive. */
    int32_t topk;
    float tau;
} lfc_config;

/* One raw frame: row-major height x width uint16 counts in device memory,
 * width and height multiples of pitch. prev, when not NULL, is the previous
 * raw frame of the series (same geometry) and enables temporal ids. */
typedef struct {
    const uint16_t *data;
    const uint16_t *prev;
    int32_t width, height, pitch;
    int32_t reserved; /* must be 0 */
} lfc_frame;

/* Creates a plan bound to cuda_stream (a cudaStream_t; NULL = legacy default
 * stream) on the current device, allocating all workspace the other calls
 * need for frames up to config->width x height and config->max_frames per
 * call. Synchronous. Errors: INVALID_ARG, NOMEM, CUDA. */
int lfc_plan_create(const lfc_config *config, void *cuda_stream, lfc_plan *out);

/* Frees the plan and its workspace after synchronising its stream. */
void lfc_plan_destroy(lfc_plan plan);

/* One-line description of the last error the plan reported. */
const char *lfc_plan_last_error(lfc_plan plan);

/* Two-dimensional image entropy criterion (Sec. 2.1.2, Eq. (1), Fig. 2c).
 * For each frame and each candidate id: the symbol stream (prediction,
 * symbol map, ordering, 16-to-8-bit realign in the id's byte layout) is
 * sorted by the first byte of every rotation only, ties in generation
 * order; adjacent bytes of the last column form 16-bit values; their
 * histogram P_t gives score = sum_t P_t * L2(P_t), L2(c) = 2^32 log2(c) in
 * fixed point (leading-bit integer part, 32 fraction bits by repeated
 * squaring in Q62). Lower entropy = higher score; the best id is the
 * highest score, ties to the lowest id.
 *   h_frames   host array of n frames (device data).
 *   d_choice   device, n bytes: best id per frame.
 *   d_scores   device, n * 256 uint64 or NULL: score of id c of frame i at
 *              [i * 256 + c]; entries of ids not judged are left untouched.
 * The pair-histogram kernel keeps per-SM scratch in the plan's workspace:
 * a plan's judge work (lfc_judge, lfc_compress, lfc_propose's judged frames,
 * replays of its batches) must not overlap on the GPU. The plan's stream
 * serialises its own calls; a batch replayed on the plan's stream keeps that
 * order too.
 * Errors: INVALID_ARG (n > max_frames, geometry beyond the plan), CUDA. */
int lfc_judge(lfc_plan plan, const lfc_frame *h_frames, int n, uint8_t *d_choice, uint64_t *d_scores);

/* Symbol stream of one frame under candidate id (Sec. 2.1.1 prediction,
 * Fig. 2a symbol image, the id's ordering): width * height uint16 symbols
 * in stream order written to d_out. Errors: INVALID_ARG, CUDA. */
int lfc_symbols(lfc_plan plan, const lfc_frame *h_frame, int id, uint16_t *d_out);

/* Bytes one frame's container can take at most (header + worst-case bzip2
 * streams of every block). block_bytes 0 selects 720000. */
size_t lfc_max_compressed_bytes(int32_t width, int32_t height, int32_t block_bytes);

/* Compresses n frames (Fig. 1c): judge (unless d_choice is given), emit the
 * chosen stream, split it into block_bytes blocks (Sec. 2.1.3) and code each
 * as a standalone level-9 bzip2 stream (RLE1, BWT of the full rotation sort,
 * MTF over the bytes in use, RUNA/RUNB zero runs, 2-6 Huffman tables chosen
 * per 50 symbols, bit packing, block CRC-32/BZIP2), then the container:
 *   0 "LFC1" | 4 u16 version 1 | 6 u16 flags (bit 0 temporal) | 8 u32 W |
 *   12 u32 H | 16 u32 pitch | 20 u8 id, 3 zero bytes | 24 u32 block_bytes |
 *   28 u32 n_blocks | 32 u32 CRC-32/BZIP2 of the raw frame bytes |
 *   36 u32 header bytes (40 + 4 n_blocks) | 40 u32 stream bytes per block |
 *   streams back to back.
 * Frame i's container is written at d_out + sum_{j<i} lfc_max_compressed_
 * bytes(W_j, H_j, block_bytes); its size goes to d_out_sizes[i].
 *   d_choice    device n ids to use, or NULL to run lfc_judge first.
 *   out_cap     bytes available at d_out; CAPACITY if below the slot sum.
 * The call blocks the host until the stream has finished the BWT rounds
 * (it reads per-round active counts). Errors: INVALID_ARG, CAPACITY, CUDA,
 * TIMEOUT (a bounded wait of the suffix sort gave up; see wait_budget_ms). */
int lfc_compress(lfc_plan plan, const lfc_frame *h_frames, int n, const uint8_t *d_choice,
                 uint8_t *d_out, size_t out_cap, uint64_t *d_out_sizes);

/* lfc_compress on frames in host memory, the containers back in host memory
 * (the whole round trip of a caller whose frames arrive on the host). Frame
 * i's data (and prev) point to host memory; they are copied to device
 * staging buffers that the plan allocates on the first call (max_frames
 * frames of the plan's size, twice when frames carry prev), then
 * compressed, and container i goes to h_out + the same offset as in
 * lfc_compress, its size to h_out_sizes[i] (host). Pinned host memory
 * makes the copies asynchronous. h_choice: host n ids, or NULL to judge.
 * Synchronous. Errors: as lfc_compress; CAPACITY if out_cap is below the
 * slot sum; NOMEM if the staging buffers cannot be allocated. */
int lfc_compress_host(lfc_plan plan, const lfc_frame *h_frames, int n, const uint8_t *h_choice, uint8_t *h_out,
                      size_t out_cap, uint64_t *h_out_sizes);

/* A batch is one lfc_compress call captured once as a CUDA graph (with the
 * suffix-sort rounds as a device-driven WHILE node), so that a stream of
 * batches with the same frame buffers and geometry costs one cudaGraphLaunch
 * each. lfc_batch_create takes the same arguments as lfc_compress, records
 * every descriptor table in a device buffer it owns (allocated here, not on
 * launch), captures the work on the plan's stream and instantiates it; it is
 * synchronous. lfc_batch_launch replays it on the plan's stream with the data
 * the frame buffers hold at that time; outputs land as for lfc_compress.
 * Batches share the plan's workspace: launches on one plan are serialised by
 * its stream. A bounded wait that gives up during a replay is reported by
 * lfc_plan_device_status. Errors: as lfc_compress, plus NOMEM, CUDA. */
typedef struct lfc_batch_s *lfc_batch;
int lfc_batch_create(lfc_plan plan, const lfc_frame *h_frames, int n, const uint8_t *d_choice, uint8_t *d_out,
                     size_t out_cap, uint64_t *d_out_sizes, lfc_batch *out);
int lfc_batch_launch(lfc_batch batch);
void lfc_batch_destroy(lfc_batch batch);

/* Standalone bzip2 streams of arbitrary byte blocks (the coder stage of
 * lfc_compress on its own). Block b is d_in[h_offsets[b] .. + h_sizes[b]),
 * 1 <= size <= 720000 and n_blocks <= the plan's block capacity
 * (lfc_plan_block_capacity). Stream b is written at d_out + b * out_stride,
 * its byte count to d_stream_sizes[b]; out_stride must be at least
 * lfc_max_stream_bytes(max size). Errors: INVALID_ARG, CAPACITY, CUDA,
 * TIMEOUT (as lfc_compress). */
int lfc_bzip2_encode(lfc_plan plan, const uint8_t *d_in, const uint64_t *h_offsets,
                     const uint32_t *h_sizes, int n_blocks, uint8_t *d_out, size_t out_stride,
                     uint32_t *d_stream_sizes);

/* The Burrows-Wheeler transform of arbitrary byte blocks exactly as the
 * coder computes it inside lfc_bzip2_encode (bzip2 format, Sec. 2.1.3): RLE1
 * of the block, then the sort of all cyclic rotations, identical rotations
 * by start index; the last column goes out. Block b is d_in[h_offsets[b] ..
 * + h_sizes[b]), 1 <= size <= 720000, n_blocks <= the plan's block capacity.
 * Its last column is written at d_L + b * L_stride (device; L_stride must
 * hold the RLE1 length bound min(900000, 5/4 size + 4)), its length (the RLE1
 * length) to d_len[b] and the row of the rotation starting at 0 to
 * d_orig[b] (both device). Used to compare the paper's first-byte judge with
 * the entropy of the real transform. Errors: INVALID_ARG, CAPACITY, CUDA,
 * TIMEOUT (as lfc_compress). */
int lfc_bwt_blocks(lfc_plan plan, const uint8_t *d_in, const uint64_t *h_offsets, const uint32_t *h_sizes,
                   int n_blocks, uint8_t *d_L, size_t L_stride, uint32_t *d_len, uint32_t *d_orig);

/* Worst-case bytes of one stream holding block_bytes input bytes. */
size_t lfc_max_stream_bytes(int32_t block_bytes);

/* Blocks one lfc_compress / lfc_bzip2_encode pass can hold. */
int lfc_plan_block_capacity(lfc_plan plan);

/* Decompresses n containers (Fig. 2b: unpack the header, bzip2-decode every
 * block, inverse predictor chosen by the header's id). Container i is
 * h_in[i] (device) of h_in_sizes[i] bytes; the frame goes to h_out[i]
 * (device), which holds h_out_bytes[i] bytes (CAPACITY below 2 * W * H of the
 * container). Temporal containers need h_prev[i] (device previous raw frame
 * of the same geometry); h_prev may be NULL when no container is temporal.
 * h_prev[i] may point at h_out[j] for j < i: frames are restored in index
 * order. Every read of a container is bounds-checked, so a corrupt container
 * returns CORRUPT (bad header, block stream, block CRC or frame CRC) and
 * never reads or writes outside the buffers. Synchronous: the host reads
 * the headers. Errors: INVALID_ARG, CAPACITY, CORRUPT, CUDA. */
int lfc_decompress(lfc_plan plan, const uint8_t *const *h_in, const uint64_t *h_in_sizes, int n,
                   uint16_t *const *h_out, const uint64_t *h_out_bytes, const uint16_t *const *h_prev);

/* Tuning knobs of the judge (an autotuner picks them per frame geometry and
 * candidate count; 0 keeps a field's default). They change only speed,
 * never results.
 *   emit_tile_lenslets      lenslets per row tile of the candidate emission
 *                           kernel: 4, 8 or 16 (default 16);
 *   chain_range_bytes       upper bound on the bytes of a candidate stream
 *                           one warp of the pair-chain kernel walks (a 32nd
 *                           per lane): 16384, 32768, 65536, 131072 or 262144
 *                           (default 262144); each launch evens the ranges
 *                           out below it so that its CTAs fill whole waves
 *                           of the device's SMs;
 *   judge_frames_per_launch frames per judge launch, 1 .. the plan's
 *                           min(max_frames, 16) (default: that maximum);
 *   wait_budget_ms          how long one bounded device wait may last
 *                           before the kernel gives up and the call returns
 *                           LFC_ERR_TIMEOUT, 1 .. 60000 (default 1000). The
 *                           suffix sort's radix passes wait on each other
 *                           (every tile waits for the digit counts of the
 *                           block's earlier tiles); such waits always end in
 *                           a correct run, so the budget only bounds a fault.
 * Errors: INVALID_ARG for values outside these sets. */
typedef struct {
    int32_t emit_tile_lenslets;
    int32_t chain_range_bytes;
    int32_t judge_frames_per_launch;
    int32_t wait_budget_ms;
} lfc_tuning;
int lfc_plan_set_tuning(lfc_plan plan, const lfc_tuning *tuning);
int lfc_plan_get_tuning(lfc_plan plan, lfc_tuning *tuning);

/* Device status of the plan's bounded waits: synchronises the plan's
 * stream and returns LFC_ERR_TIMEOUT if a device wait has given up since the
 * last call (for example in a replayed batch, whose launch returns before the
 * GPU runs it), clearing that state; LFC_OK otherwise. lfc_compress and
 * lfc_bzip2_encode report a wait that gives up in their own calls (they read
 * the suffix sort's state) and start from a clear state. Errors: CUDA. */
int lfc_plan_device_status(lfc_plan plan);

/* Fault injection for tests of the bounded waits (host side: nothing on the
 * GPU faults). LFC_FAULT_SORT_WITHHOLD: in the next suffix sort the first
 * tile of the first block sorts its elements but never publishes its digit
 * counts, so the block's later tiles wait for a flag that nothing sets, give
 * up after the plan's wait budget and the call returns LFC_ERR_TIMEOUT
 * (its output is void). The fault is set on the device, asynchronously on
 * the plan's stream, and fires in the next suffix sort that runs there (an
 * lfc_compress, lfc_bzip2_encode or batch replay), once; the plan stays
 * usable. LFC_FAULT_NONE cancels a pending fault. Errors: INVALID_ARG, CUDA. */
enum { LFC_FAULT_NONE = 0, LFC_FAULT_SORT_WITHHOLD = 1 };
int lfc_plan_inject_fault(lfc_plan plan, int fault);

/* Stage timing (tracing). With timing enabled the plan records CUDA events on
 * its stream around each stage below and accumulates their device time; the
 * counters only change while enabled. lfc_plan_set_timing also zeroes them.
 * lfc_plan_timing synchronises the plan's stream, then writes n_stages
 * accumulated milliseconds to ms (host) and span counts to spans (host, may
 * be NULL). Errors: INVALID_ARG, CUDA. */
enum {
    LFC_STAGE_JUDGE_HIST = 0, /* judge-BWT pair histograms (one kernel) */
    LFC_STAGE_JUDGE_SCORE,    /* segment fixup, entropy scores, argmax */
    LFC_STAGE_EMIT,           /* chosen symbol streams */
    LFC_STAGE_CRC,            /* raw-frame and block CRCs */
    LFC_STAGE_RLE1,
    LFC_STAGE_BWT_SORT8,      /* 8-byte prefix radix sort: the 8 LSD passes */
    LFC_STAGE_BWT_REFINE,     /* prefix-doubling rounds */
    LFC_STAGE_BWT_OUT,        /* last column, origin, bytes in use */
    LFC_STAGE_MTF,            /* MTF and RUNA/RUNB coding */
    LFC_STAGE_HUFFMAN,
    LFC_STAGE_PACK,
    LFC_STAGE_CONTAINER,
    LFC_STAGE_JUDGE_EMIT,     /* every candidate stream of the judged frames */
    LFC_STAGE_BWT_KEYS,       /* prefix keys, byte histograms, sort work items */
    LFC_NUM_STAGES
};
int lfc_plan_set_timing(lfc_plan plan, int enable);
int lfc_plan_timing(lfc_plan plan, double *ms, int64_t *spans, int n_stages);

/* Kernel launches this plan has issued since creation (host counter). */
int64_t lfc_plan_launch_count(lfc_plan plan);

/* Suffix-sort counters since creation (host values, read without a sync):
 * out[0] BWT calls, out[1] prefix-doubling rounds, out[2] elements sorted
 * (sum of RLE1 block lengths; exact after the stream is synchronised),
 * out[3] tied elements entering rounds (sum over rounds), out[4 + r] tied
 * elements entering round r (r < n - 4, summed over calls). Returns the
 * number of values written. */
int lfc_plan_bwt_counters(lfc_plan plan, int64_t *out, int n);

/* Allocation-free judge of one frame. The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory, such
 * as an acquisition loop that reserves its whole device-memory budget at
 * start-up, or a plug-in running inside another framework whose allocator
 * owns the device, where cudaMalloc/cudaFree (which can also synchronise
 * the device) are not allowed on the processing path. It needs no plan and
 * calls no allocating routine: its scratch (one 65536-bin histogram, chain
 * summaries, the log2 table, descriptors and scores; about 0.8 MB) is one
 * file-scope device array that every GPU loading the library holds until
 * the process exits. Same results as lfc_judge for one frame:
 *   h_frame    host pointer to one frame (device data); at most 4096 rows,
 *              width at most 2656, 2 * width * height <= 2^26;
 *   h_ids      host array of n_ids (1..256) valid candidate ids; temporal
 *              ids need h_frame->prev;
 *   d_choice   device, 1 byte: the best id;
 *   d_scores   device, 256 uint64 or NULL: score of id c at [c] for the
 *              judged ids, other entries untouched;
 *   cuda_stream the stream to run on (NULL = legacy default stream).
 * The first call on a device looks up the array's device address, which
 * loads the library's device code on that device if it is not loaded yet;
 * make that first call before any stream capture. Every call looks the
 * address up again (it changes when the device's context is re-created, e.g.
 * after cudaDeviceReset) and launches a small kernel that rebuilds the log2
 * table when the array does not hold it yet (the array starts zeroed in
 * every new context); no call synchronises. All calls share the one array
 * and leave their contents in it; each call clears what must start at zero,
 * and calls whose work overlaps on the GPU (other streams, other host
 * threads) race on it. If a CUDA error from earlier work is pending on the
 * calling thread, the call returns CUDA without launching anything and
 * leaves that error in place. Errors: INVALID_ARG (sizes beyond the limits
 * above, bad ids), CUDA. */
int lfc_judge_noalloc(const lfc_frame *h_frame, const uint8_t *h_ids, int n_ids, uint8_t *d_choice,
                      uint64_t *d_scores, void *cuda_stream);

/* Learned candidate proposal (a small network trained to predict the
 * criterion's choice; the paper motivates cutting the criterion's time,
 * Sec. 4). Input: a 2 x 256 x 256 thumbnail (channel 0 raw layout, channel 1
 * view-major mosaic; bs x bs block means with bs = ceil(max(W, H) / 256),
 * edge blocks over their valid pixels; log1p(max(mean - 100, 0)) / 8;
 * zero padding). Network: 4 x [3x3 convolution (2 -> 32, then 32 -> 32
 * channels), zero padding 1, bias, ReLU], mean pool, linear 32 -> K, softmax.
 * BF16 weights and activations, FP32 accumulation (tensor cores), FP32 master
 * parameters and Adam state. Parameters (FP32, this order): for l = 0..3
 * w_l[3][3][cin_l][32] (cin = 2, 32, 32, 32) then b_l[32]; wl[32][K]; bl[K].
 * All calls run on the stream given at creation; d_* are device pointers. */
typedef struct lfc_cnn_s *lfc_cnn;
/* Allocates the network for n_classes outputs (2..64) and batches up to
 * max_batch, initialised He-normal from seed. Synchronous. */
int lfc_cnn_create(int n_classes, int max_batch, uint64_t seed, void *cuda_stream, lfc_cnn *out);
void lfc_cnn_destroy(lfc_cnn cnn);
const char *lfc_cnn_last_error(lfc_cnn cnn);
size_t lfc_cnn_param_count(lfc_cnn cnn);
/* Host FP32 parameters in / out (checkpoints); get also returns the last
 * gradients when h_grads is not NULL. Synchronous. */
int lfc_cnn_set_params(lfc_cnn cnn, const float *h_params, size_t n);
int lfc_cnn_get_params(lfc_cnn cnn, float *h_params, float *h_grads, size_t n);
/* Thumbnails of n frames (prev ignored) into the network's input;
 * d_thumbs (n x 2 x 256 x 256 FP32) receives a copy when not NULL. */
int lfc_cnn_thumbnails(lfc_cnn cnn, const lfc_frame *h_frames, int n, float *d_thumbs);
/* Input from caller FP32 thumbnails (n x 2 x 256 x 256), rounded to BF16. */
int lfc_cnn_set_thumbnails(lfc_cnn cnn, const float *d_thumbs, int n);
/* Softmax probabilities (n x K FP32) of the current input. */
int lfc_cnn_forward(lfc_cnn cnn, int n, float *d_probs);
/* Forward, mean cross-entropy with d_labels (n int32 class indices) and the
 * gradients of every parameter; per-frame losses to d_loss if not NULL. */
int lfc_cnn_backward(lfc_cnn cnn, int n, const int32_t *d_labels, float *d_loss);
/* One Adam update with the last gradients (bias-corrected). */
int lfc_cnn_adam_step(lfc_cnn cnn, float lr, float beta1, float beta2, float eps);

/* Attaches a trained network to a plan: class k of the network is candidate
 * id h_class_ids[k] (n_classes must equal the network's). With topk > 0 the
 * judge of every frame without a previous frame runs only on the network's
 * topk most probable ids, or on all candidates when the top probability is
 * below tau; temporal frames are always judged exhaustively. The network
 * must run on the plan's stream. cnn = NULL detaches. */
int lfc_plan_set_proposal(lfc_plan plan, lfc_cnn cnn, const uint8_t *h_class_ids, int n_classes, int topk, float tau);

/* Candidate masks the proposal gives n frames (n x 4 uint64, bit id % 64 of
 * word id / 64), as used by lfc_judge/lfc_compress. Errors: INVALID_ARG when
 * no network is attached. */
int lfc_propose(lfc_plan plan, const lfc_frame *h_frames, int n, uint64_t *d_masks);

/* Text of a status code. */
const char *lfc_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* LFC_H */

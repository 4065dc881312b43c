// api.cu -- the C ABI of liblfc (include/lfc.h): plans, workspace, and the
// order of the stages (Fig. 1c: prediction, entropy criterion, block bzip2
// coding, header packing). All compute runs in the kernels of this library.
#include "lfc_common.cuh"

#include <algorithm>
#include <cstring>
#include <new>

using namespace lfc;

namespace {

constexpr int kJudgeFramesCap = 8;

int fail(lfc_plan P, int code, const std::string &what, cudaError_t e = cudaSuccess) {
    if (P) {
        P->err = what;
        if (e != cudaSuccess) {
            P->err += ": ";
            P->err += cudaGetErrorString(e);
        }
    }
    return code;
}

#define CK(x)                                                              \
    do {                                                                   \
        cudaError_t _e = (x);                                              \
        if (_e != cudaSuccess) return fail(P, LFC_ERR_CUDA, #x, _e);       \
    } while (0)

bool id_valid(int id) {
    const int f = id & 15, dom = (id >> 4) & 3;
    return id >= 0 && id < 256 && f <= 7 && dom <= 2 && !(f == 0 && dom != 0);
}

int64_t stream_bound(int64_t L) {
    const int64_t m = L + L / 4 + 4;
    const int64_t nmtf = m + 1;
    const int64_t nsel = (nmtf + 49) / 50;
    const int64_t bits = 427 + 6 * nsel + 6 * (5 + 258 * 33) + 17 * nmtf + 87;
    return (bits + 7) / 8 + 16;
}

int64_t container_bound(int64_t W, int64_t H, int64_t bb) {
    const int64_t n = 2 * W * H;
    const int64_t nb = (n + bb - 1) / bb;
    int64_t t = 40 + 4 * nb + (nb - 1) * stream_bound(bb) + stream_bound(n - (nb - 1) * bb);
    return (t + 255) & ~(int64_t)255;
}

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
    return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T) + 256);
}

bool geometry_ok(int W, int H, int p) {
    return W > 0 && H > 0 && p > 0 && W % p == 0 && H % p == 0 && (int64_t)W * H * 2 <= ((int64_t)1 << 26);
}

int check_frame(lfc_plan P, const lfc_frame &f) {
    if (!f.data) return fail(P, LFC_ERR_INVALID_ARG, "frame data is NULL");
    if (!geometry_ok(f.width, f.height, f.pitch)) return fail(P, LFC_ERR_INVALID_ARG, "frame geometry invalid");
    if ((int64_t)f.width * f.height > (int64_t)P->cfg.width * P->cfg.height || f.width > P->cfg.width)
        return fail(P, LFC_ERR_INVALID_ARG, "frame larger than the plan");
    if (f.reserved != 0) return fail(P, LFC_ERR_INVALID_ARG, "lfc_frame.reserved must be 0");
    return LFC_OK;
}

FrameDev to_dev(const lfc_frame &f, bool temporal_ok) {
    FrameDev d;
    d.X = f.data;
    d.prev = temporal_ok ? f.prev : nullptr;
    d.W = f.width;
    d.H = f.height;
    d.p = f.pitch;
    d.Nx = f.width / f.pitch;
    d.Ny = f.height / f.pitch;
    return d;
}

int block_bytes_of(lfc_plan P) { return P->cfg.block_bytes > 0 ? P->cfg.block_bytes : kMaxBlockBytes; }

}  // namespace

// ---------------------------------------------------------------- tracing
namespace lfc {
static cudaEvent_t take_event(lfc_plan P) {
    if (!P->event_pool.empty()) {
        cudaEvent_t e = P->event_pool.back();
        P->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void stage_begin(lfc_plan P, int stage) {
    if (!P->timing) return;
    cudaEvent_t e = take_event(P);
    cudaEventRecord(e, P->stream);
    P->open_ev[stage] = e;
}

void stage_end(lfc_plan P, int stage) {
    if (!P->timing || !P->open_ev[stage]) return;
    cudaEvent_t e = take_event(P);
    cudaEventRecord(e, P->stream);
    P->spans.push_back({stage, P->open_ev[stage], e});
    P->open_ev[stage] = nullptr;
}
}  // namespace lfc

static cudaError_t harvest(lfc_plan P) {
    cudaError_t e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return e;
    for (auto &sp : P->spans) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sp.a, sp.b) == cudaSuccess) {
            P->stage_ms[sp.stage] += ms;
            P->stage_spans[sp.stage] += 1;
        }
        P->event_pool.push_back(sp.a);
        P->event_pool.push_back(sp.b);
    }
    P->spans.clear();
    return cudaSuccess;
}

extern "C" int lfc_plan_set_timing(lfc_plan P, int enable) {
    if (!P) return LFC_ERR_INVALID_ARG;
    CK(harvest(P));
    for (int i = 0; i < LFC_NUM_STAGES; i++) { P->stage_ms[i] = 0; P->stage_spans[i] = 0; }
    P->timing = enable != 0;
    return LFC_OK;
}

extern "C" int lfc_plan_timing(lfc_plan P, double *ms, int64_t *spans, int n_stages) {
    if (!P || !ms || n_stages < 0) return LFC_ERR_INVALID_ARG;
    CK(harvest(P));
    for (int i = 0; i < n_stages && i < LFC_NUM_STAGES; i++) {
        ms[i] = P->stage_ms[i];
        if (spans) spans[i] = P->stage_spans[i];
    }
    return LFC_OK;
}

extern "C" int64_t lfc_plan_launch_count(lfc_plan P) { return P ? P->launches : 0; }

extern "C" const char *lfc_status_string(int s) {
    switch (s) {
    case LFC_OK: return "ok";
    case LFC_ERR_INVALID_ARG: return "invalid argument";
    case LFC_ERR_CAPACITY: return "output capacity too small";
    case LFC_ERR_CORRUPT: return "corrupt input";
    case LFC_ERR_CUDA: return "CUDA error";
    case LFC_ERR_TIMEOUT: return "device wait timed out";
    case LFC_ERR_UNIMPLEMENTED: return "not implemented";
    case LFC_ERR_NOMEM: return "out of device memory";
    default: return "unknown status";
    }
}

extern "C" size_t lfc_max_stream_bytes(int32_t block_bytes) {
    if (block_bytes <= 0 || block_bytes > kMaxBlockBytes) block_bytes = kMaxBlockBytes;
    return (size_t)stream_bound(block_bytes);
}

extern "C" size_t lfc_max_compressed_bytes(int32_t width, int32_t height, int32_t block_bytes) {
    if (width <= 0 || height <= 0) return 0;
    if (block_bytes <= 0 || block_bytes > kMaxBlockBytes) block_bytes = kMaxBlockBytes;
    return (size_t)container_bound(width, height, block_bytes);
}

extern "C" const char *lfc_plan_last_error(lfc_plan P) { return P ? P->err.c_str() : "null plan"; }

extern "C" int lfc_plan_block_capacity(lfc_plan P) { return P ? P->block_cap : 0; }

static void free_ws(Workspace &w) {
    void *ptrs[] = {w.hist, w.summ, w.scores, w.choice, w.jframes, w.cand, w.l2tab, w.stream, w.blocks, w.bstate,
                    w.rle, w.sa, w.sa2, w.rank, w.act, w.act2, w.val, w.val2, w.tilecnt, w.tileaux, w.bwt,
                    w.mtfidx, w.mtflists, w.mtfrec, w.mtfreclen, w.sym, w.freq, w.sel, w.lens, w.codes, w.packed, w.cstream, w.chain_first,
                    w.act_total, w.block_dst, w.frame_crc, w.crc_part, w.chunk_desc, w.dec_tt};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (w.h_act_total) cudaFreeHost(w.h_act_total);
    w = Workspace();
}

extern "C" int lfc_plan_create(const lfc_config *cfg, void *cuda_stream, lfc_plan *out) {
    if (!cfg || !out) return LFC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!geometry_ok(cfg->width, cfg->height, cfg->pitch) || cfg->max_frames < 1) return LFC_ERR_INVALID_ARG;
    if (cfg->block_bytes < 0 || cfg->block_bytes > kMaxBlockBytes) return LFC_ERR_INVALID_ARG;
    if (cfg->pitch > 64) return LFC_ERR_INVALID_ARG;
    lfc_plan P = new (std::nothrow) lfc_plan_s();
    if (!P) return LFC_ERR_NOMEM;
    P->cfg = *cfg;
    if (P->cfg.keyframe_interval <= 0) P->cfg.keyframe_interval = 16;
    P->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&P->device);
    // candidate ids
    bool any = false;
    for (int i = 0; i < 4; i++) any |= cfg->candidate_mask[i] != 0;
    if (!any) {
        for (int o = 0; o < 2; o++) {
            P->ids_spatial.push_back(LFC_ID(0, 0, o, 0));
            for (int d = 0; d < 3; d++)
                for (int f = 4; f <= 7; f++) P->ids_spatial.push_back(LFC_ID(f, d, o, 0));
        }
        std::sort(P->ids_spatial.begin(), P->ids_spatial.end());
        if (cfg->temporal)
            for (uint8_t id : P->ids_spatial) P->ids_temporal.push_back((uint8_t)(id | 0x80));
    } else {
        for (int id = 0; id < 256; id++) {
            if (!((cfg->candidate_mask[id >> 6] >> (id & 63)) & 1)) continue;
            if (!id_valid(id)) { delete P; return LFC_ERR_INVALID_ARG; }
            if (id & 0x80) {
                if (cfg->temporal) P->ids_temporal.push_back((uint8_t)id);
            } else {
                P->ids_spatial.push_back((uint8_t)id);
            }
        }
        if (P->ids_spatial.empty()) { delete P; return LFC_ERR_INVALID_ARG; }
    }
    const int K = (int)(P->ids_spatial.size() + P->ids_temporal.size());
    if (K > kMaxCand) { delete P; return LFC_ERR_INVALID_ARG; }

    Workspace &ws = P->ws;
    const int F = cfg->max_frames;
    const int64_t n_max = 2LL * cfg->width * cfg->height;
    const int bb = block_bytes_of(P);
    const int64_t bpf = (n_max + bb - 1) / bb;
    P->judge_frames_cap = std::min(F, kJudgeFramesCap);
    P->block_cap = (int)std::max<int64_t>(bpf, std::min<int64_t>((int64_t)F * bpf, 192));
    const int JF = P->judge_frames_cap, BC = P->block_cap;
    const int64_t segs_max = (n_max + chain_seg_bytes() - 1) / chain_seg_bytes();
    ws.summ_cap = (int64_t)JF * kMaxCand * segs_max;
    ws.cstream_kmax = K;
    ws.cstream_slot = (n_max + 255) & ~(int64_t)255;
    ws.stream_slot = (n_max + 255) & ~(int64_t)255;
    ws.stream_words = (stream_bound(bb) + 3) / 4 + 4;
    ws.crc_part_cap = 262144;
    ws.chunk_desc_bytes = 8u << 20;
    cudaError_t e = cudaSuccess;
#define AL(ptr, count)                                           \
    if (e == cudaSuccess) e = dalloc(&ws.ptr, (size_t)(count));
    AL(hist, (size_t)JF * kMaxCand * kHistBins);
    AL(summ, (size_t)ws.summ_cap * 512);
    AL(scores, (size_t)F * 256);
    AL(choice, (size_t)F);
    AL(jframes, (size_t)JF);
    AL(cand, (size_t)1 << 20);
    AL(l2tab, (size_t)kHistBins);
    AL(stream, (size_t)F * ws.stream_slot);
    AL(cstream, (size_t)JF * K * ws.cstream_slot);
    AL(chain_first, (size_t)ws.summ_cap * chain_first_bytes_per_cta());
    AL(blocks, (size_t)BC);
    AL(bstate, (size_t)BC);
    AL(rle, (size_t)BC * kBlockCap);
    AL(sa, (size_t)BC * kBlockCap);
    AL(sa2, (size_t)BC * kBlockCap);
    AL(rank, (size_t)BC * kBlockCap);
    AL(act, (size_t)BC * kBlockCap);
    AL(act2, (size_t)BC * kBlockCap);
    AL(val, (size_t)BC * kBlockCap);
    AL(val2, (size_t)BC * kBlockCap);
    AL(tilecnt, (size_t)BC * 256 * kTilesPerBlock);
    AL(tileaux, (size_t)BC * kTilesPerBlock * 4);
    AL(bwt, (size_t)BC * kBlockCap);
    AL(mtfidx, (size_t)BC * kBlockCap);
    AL(mtflists, (size_t)BC * kTilesPerBlock * 256);
    AL(mtfrec, (size_t)BC * kTilesPerBlock * 256);
    AL(mtfreclen, (size_t)BC * kTilesPerBlock);
    AL(sym, (size_t)BC * (kBlockCap + 64));
    AL(freq, (size_t)BC * kMaxAlpha);
    AL(sel, (size_t)BC * kMaxSelectors);
    AL(lens, (size_t)BC * kMaxGroups * kMaxAlpha);
    AL(codes, (size_t)BC * kMaxGroups * kMaxAlpha);
    AL(packed, (size_t)BC * ws.stream_words);
    AL(act_total, (size_t)4);
    AL(block_dst, (size_t)BC);
    AL(frame_crc, (size_t)F);
    AL(crc_part, (size_t)ws.crc_part_cap);
#undef AL
    if (e == cudaSuccess) e = cudaMalloc(&ws.chunk_desc, ws.chunk_desc_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&ws.h_act_total), 4 * sizeof(int32_t));
    if (e == cudaSuccess) e = init_l2_table(ws.l2tab, P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        free_ws(ws);
        delete P;
        return oom ? LFC_ERR_NOMEM : LFC_ERR_CUDA;
    }
    *out = P;
    return LFC_OK;
}

extern "C" void lfc_plan_destroy(lfc_plan P) {
    if (!P) return;
    cudaStreamSynchronize(P->stream);
    harvest(P);
    for (cudaEvent_t e : P->event_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : P->open_ev)
        if (e) cudaEventDestroy(e);
    free_ws(P->ws);
    delete P;
}

// ------------------------------------------------------------------ judge
static int judge_impl(lfc_plan P, const lfc_frame *frames, int n, uint8_t *d_choice, uint64_t *d_scores) {
    Workspace &ws = P->ws;
    const int64_t seg_bytes = chain_seg_bytes();
    for (int f0 = 0; f0 < n; f0 += P->judge_frames_cap) {
        const int f1 = std::min(n, f0 + P->judge_frames_cap);
        const int nf = f1 - f0;
        std::vector<JudgeFrame> jf(nf);
        std::vector<int32_t> frame_index(nf), hist_frame;
        std::vector<uint8_t> cand;
        int64_t cta = 0, hist = 0, summ = 0;
        JudgeLaunch L{0, 16, 0, 0, 0};
        for (int i = 0; i < nf; i++) {
            const lfc_frame &fr = frames[f0 + i];
            const bool tmp = fr.prev != nullptr && !P->ids_temporal.empty();
            JudgeFrame &J = jf[i];
            J.F = to_dev(fr, tmp);
            J.cand_off = (int32_t)cand.size();
            uint32_t fset[2] = {0, 0};
            for (uint8_t id : P->ids_spatial) cand.push_back(id);
            if (tmp)
                for (uint8_t id : P->ids_temporal) cand.push_back(id);
            for (size_t k = J.cand_off; k < cand.size(); k++) {
                const int id = cand[k], f = id & 15, dom = (id >> 4) & 3;
                if (f && dom != 1) fset[(id >> 7) & 1] |= 1u << f;
            }
            L.nslots_max = std::max(L.nslots_max, std::max(__builtin_popcount(fset[0]), __builtin_popcount(fset[1])));
            L.any_temporal |= tmp ? 1 : 0;
            L.max_p = std::max(L.max_p, fr.pitch);
            J.K = (int32_t)(cand.size() - J.cand_off);
            const int64_t nbytes = 2LL * fr.width * fr.height;
            J.rows_per_seg = 0;
            J.segs = (int32_t)((nbytes + seg_bytes - 1) / seg_bytes);
            J.cta_base = cta;
            J.hist_off = hist;
            J.summ_off = summ;
            cta += (int64_t)J.K * J.segs;
            summ += (int64_t)J.K * J.segs;
            for (int k = 0; k < J.K; k++) hist_frame.push_back(i);
            hist += J.K;
            frame_index[i] = f0 + i;
        }
        // lenslets per emission tile: as many as shared memory allows (<= 16)
        L.TS = 16;
        while (L.TS > 1 && emit_all_smem_bytes(L.max_p, L.TS, L.nslots_max) > 200 * 1024) L.TS /= 2;
        if (emit_all_smem_bytes(L.max_p, L.TS, L.nslots_max) > 200 * 1024)
            return fail(P, LFC_ERR_INVALID_ARG, "pitch too large for the emission tile");
        for (int i = 0; i < nf; i++) {
            const FrameDev &F = jf[i].F;
            L.max_tiles = std::max(L.max_tiles, F.Ny * ((F.Nx + L.TS - 1) / L.TS));
        }
        if (summ > ws.summ_cap) return fail(P, LFC_ERR_INVALID_ARG, "judge summary capacity exceeded");
        // one staging blob: frames | frame_index | hist_frame | cand
        const size_t o1 = sizeof(JudgeFrame) * nf;
        const size_t o2 = o1 + 4 * nf;
        const size_t o3 = o2 + 4 * hist_frame.size();
        const size_t total = o3 + cand.size();
        if (total > ((size_t)1 << 20)) return fail(P, LFC_ERR_INVALID_ARG, "judge table too large");
        std::vector<uint8_t> blob(total);
        memcpy(blob.data(), jf.data(), o1);
        memcpy(blob.data() + o1, frame_index.data(), 4 * nf);
        memcpy(blob.data() + o2, hist_frame.data(), 4 * hist_frame.size());
        memcpy(blob.data() + o3, cand.data(), cand.size());
        uint8_t *d = reinterpret_cast<uint8_t *>(ws.cand);
        CK(cudaMemcpyAsync(d, blob.data(), total, cudaMemcpyHostToDevice, P->stream));
        CK(launch_judge(P, reinterpret_cast<const JudgeFrame *>(d), nf, cta, L, d + o3, hist, d_scores, d_choice));
    }
    return LFC_OK;
}

extern "C" int lfc_judge(lfc_plan P, const lfc_frame *frames, int n, uint8_t *d_choice, uint64_t *d_scores) {
    if (!P || !frames || n < 1 || !d_choice) return fail(P, LFC_ERR_INVALID_ARG, "lfc_judge: bad arguments");
    if (n > P->cfg.max_frames) return fail(P, LFC_ERR_INVALID_ARG, "lfc_judge: n > max_frames");
    for (int i = 0; i < n; i++) {
        int r = check_frame(P, frames[i]);
        if (r) return r;
    }
    return judge_impl(P, frames, n, d_choice, d_scores ? d_scores : P->ws.scores);
}

extern "C" int lfc_symbols(lfc_plan P, const lfc_frame *frame, int id, uint16_t *d_out) {
    if (!P || !frame || !d_out) return fail(P, LFC_ERR_INVALID_ARG, "lfc_symbols: bad arguments");
    int r = check_frame(P, *frame);
    if (r) return r;
    if (!id_valid(id)) return fail(P, LFC_ERR_INVALID_ARG, "lfc_symbols: invalid id");
    if ((id & 0x80) && !frame->prev) return fail(P, LFC_ERR_INVALID_ARG, "lfc_symbols: temporal id needs prev");
    CK(launch_symbols_one(to_dev(*frame, (id & 0x80) != 0), id, d_out, P->stream));
    count_launches(P, 1);
    return LFC_OK;
}

// ------------------------------------------------------------------ coder
// Runs the coder on blocks[0..nb) of the plan's block table (already staged).
static int code_blocks(lfc_plan P, const std::vector<BlockDesc> &blocks) {
    Workspace &ws = P->ws;
    const int nb = (int)blocks.size();
    int max_len = 0;
    for (const BlockDesc &b : blocks) max_len = std::max(max_len, b.len);
    CK(cudaMemcpyAsync(ws.blocks, blocks.data(), sizeof(BlockDesc) * nb, cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemsetAsync(ws.bstate, 0, sizeof(BlockState) * nb, P->stream));
    stage_begin(P, LFC_STAGE_CRC);
    CK(launch_block_crc(P, blocks.data(), nb, ws.bstate));
    stage_end(P, LFC_STAGE_CRC);
    stage_begin(P, LFC_STAGE_RLE1);
    CK(launch_rle1(P, nb));
    stage_end(P, LFC_STAGE_RLE1);
    const int max_m = std::min(kRleCap, max_len + max_len / 4 + 4);
    CK(launch_bwt(P, nb, max_m));
    stage_begin(P, LFC_STAGE_MTF);
    CK(launch_mtf_rle2(P, nb));
    stage_end(P, LFC_STAGE_MTF);
    stage_begin(P, LFC_STAGE_HUFFMAN);
    CK(launch_huffman(P, nb));
    stage_end(P, LFC_STAGE_HUFFMAN);
    stage_begin(P, LFC_STAGE_PACK);
    CK(launch_pack(P, nb));
    stage_end(P, LFC_STAGE_PACK);
    return LFC_OK;
}

extern "C" int lfc_bzip2_encode(lfc_plan P, const uint8_t *d_in, const uint64_t *h_offsets, const uint32_t *h_sizes,
                                int n_blocks, uint8_t *d_out, size_t out_stride, uint32_t *d_stream_sizes) {
    if (!P || !d_in || !h_offsets || !h_sizes || !d_out || !d_stream_sizes || n_blocks < 1)
        return fail(P, LFC_ERR_INVALID_ARG, "lfc_bzip2_encode: bad arguments");
    if (n_blocks > P->block_cap) return fail(P, LFC_ERR_INVALID_ARG, "lfc_bzip2_encode: too many blocks");
    std::vector<BlockDesc> blocks(n_blocks);
    uint32_t max_size = 0;
    for (int b = 0; b < n_blocks; b++) {
        if (h_sizes[b] < 1 || h_sizes[b] > (uint32_t)kMaxBlockBytes)
            return fail(P, LFC_ERR_INVALID_ARG, "lfc_bzip2_encode: block size outside 1..720000");
        blocks[b].src = d_in + h_offsets[b];
        blocks[b].len = (int32_t)h_sizes[b];
        blocks[b].frame = -1;
        max_size = std::max(max_size, h_sizes[b]);
    }
    if (out_stride < (size_t)stream_bound(max_size)) return fail(P, LFC_ERR_CAPACITY, "lfc_bzip2_encode: out_stride too small");
    int r = code_blocks(P, blocks);
    if (r) return r;
    stage_begin(P, LFC_STAGE_CONTAINER);
    CK(launch_copy_streams(P, n_blocks, d_out, out_stride, d_stream_sizes));
    stage_end(P, LFC_STAGE_CONTAINER);
    return LFC_OK;
}

extern "C" int lfc_compress(lfc_plan P, const lfc_frame *frames, int n, const uint8_t *d_choice, uint8_t *d_out,
                            size_t out_cap, uint64_t *d_out_sizes) {
    if (!P || !frames || n < 1 || !d_out || !d_out_sizes) return fail(P, LFC_ERR_INVALID_ARG, "lfc_compress: bad arguments");
    if (n > P->cfg.max_frames) return fail(P, LFC_ERR_INVALID_ARG, "lfc_compress: n > max_frames");
    Workspace &ws = P->ws;
    const int bb = block_bytes_of(P);
    std::vector<uint64_t> out_off(n);
    uint64_t need = 0;
    for (int i = 0; i < n; i++) {
        int r = check_frame(P, frames[i]);
        if (r) return r;
        out_off[i] = need;
        need += container_bound(frames[i].width, frames[i].height, bb);
    }
    if (need > out_cap) return fail(P, LFC_ERR_CAPACITY, "lfc_compress: out_cap below the sum of container bounds");
    const uint8_t *choice = d_choice;
    if (!choice) {
        int r = judge_impl(P, frames, n, ws.choice, ws.scores);
        if (r) return r;
        choice = ws.choice;
    }
    std::vector<FrameDev> fd(n);
    std::vector<uint8_t *> dst(n);
    std::vector<const uint8_t *> raw(n);
    std::vector<int64_t> rawlen(n);
    for (int i = 0; i < n; i++) {
        fd[i] = to_dev(frames[i], frames[i].prev != nullptr);
        dst[i] = ws.stream + (size_t)i * ws.stream_slot;
        raw[i] = reinterpret_cast<const uint8_t *>(frames[i].data);
        rawlen[i] = 2LL * frames[i].width * frames[i].height;
    }
    stage_begin(P, LFC_STAGE_EMIT);
    CK(launch_emit(fd.data(), choice, n, dst.data(), P->stream));
    count_launches(P, (n + 7) / 8);
    stage_end(P, LFC_STAGE_EMIT);
    stage_begin(P, LFC_STAGE_CRC);
    CK(launch_range_crc(P, raw.data(), rawlen.data(), n, ws.frame_crc));
    stage_end(P, LFC_STAGE_CRC);
    // passes of whole frames
    int f0 = 0;
    while (f0 < n) {
        std::vector<BlockDesc> blocks;
        std::vector<int32_t> block0;
        int f1 = f0;
        while (f1 < n) {
            const int64_t nbytes = rawlen[f1];
            const int64_t nbf = (nbytes + bb - 1) / bb;
            if ((int64_t)blocks.size() + nbf > P->block_cap) break;
            block0.push_back((int32_t)blocks.size());
            for (int64_t k = 0; k < nbf; k++) {
                BlockDesc d;
                d.src = dst[f1] + k * bb;
                d.len = (int32_t)std::min<int64_t>(bb, nbytes - k * bb);
                d.frame = f1;
                blocks.push_back(d);
            }
            f1++;
        }
        if (f1 == f0) return fail(P, LFC_ERR_INVALID_ARG, "lfc_compress: frame needs more blocks than the plan holds");
        block0.push_back((int32_t)blocks.size());
        int r = code_blocks(P, blocks);
        if (r) return r;
        stage_begin(P, LFC_STAGE_CONTAINER);
        CK(launch_container(P, f1 - f0, block0.data(), fd.data() + f0, choice + f0, ws.frame_crc + f0, d_out,
                            out_off.data() + f0, d_out_sizes + f0, bb));
        stage_end(P, LFC_STAGE_CONTAINER);
        f0 = f1;
    }
    return LFC_OK;
}

static uint32_t rd32h(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

extern "C" int lfc_decompress(lfc_plan P, const uint8_t *const *h_in, const uint64_t *h_in_sizes, int n,
                              uint16_t *const *h_out, const uint64_t *h_out_bytes, const uint16_t *const *h_prev) {
    if (!P || !h_in || !h_in_sizes || !h_out || !h_out_bytes || n < 1)
        return fail(P, LFC_ERR_INVALID_ARG, "lfc_decompress: bad arguments");
    if (n > P->cfg.max_frames) return fail(P, LFC_ERR_INVALID_ARG, "lfc_decompress: n > max_frames");
    Workspace &ws = P->ws;
    struct Hdr { int W, H, p, id, bb, nb; uint32_t crc; std::vector<uint32_t> sizes; };
    std::vector<Hdr> hd(n);
    // headers: the host reads them (two small synchronous copies per container)
    for (int i = 0; i < n; i++) {
        if (!h_in[i] || !h_out[i]) return fail(P, LFC_ERR_INVALID_ARG, "lfc_decompress: NULL buffer");
        if (h_in_sizes[i] < 40) return fail(P, LFC_ERR_CORRUPT, "container shorter than its header");
        uint8_t h[40];
        CK(cudaMemcpyAsync(h, h_in[i], 40, cudaMemcpyDeviceToHost, P->stream));
        CK(cudaStreamSynchronize(P->stream));
        Hdr &H = hd[i];
        if (memcmp(h, "LFC1", 4) != 0 || h[4] != 1 || h[5] != 0) return fail(P, LFC_ERR_CORRUPT, "bad magic or version");
        H.W = (int)rd32h(h + 8);
        H.H = (int)rd32h(h + 12);
        H.p = (int)rd32h(h + 16);
        H.id = h[20];
        H.bb = (int)rd32h(h + 24);
        H.nb = (int)rd32h(h + 28);
        H.crc = rd32h(h + 32);
        const uint32_t hdr = rd32h(h + 36);
        if (rd32h(h + 8) > 65536 || rd32h(h + 12) > 65536 || !geometry_ok(H.W, H.H, H.p) || !id_valid(H.id))
            return fail(P, LFC_ERR_CORRUPT, "bad geometry or id");
        if ((int64_t)H.W * H.H > (int64_t)P->cfg.width * P->cfg.height || H.W > P->cfg.width)
            return fail(P, LFC_ERR_INVALID_ARG, "container frame larger than the plan");
        if (((h[6] & 1) != 0) != ((H.id & 0x80) != 0) || h[7] != 0 || h[21] || h[22] || h[23])
            return fail(P, LFC_ERR_CORRUPT, "bad flags");
        if (H.bb < 1 || H.bb > kMaxBlockBytes) return fail(P, LFC_ERR_CORRUPT, "bad block size");
        const int64_t nbytes = 2LL * H.W * H.H;
        if (H.nb != (nbytes + H.bb - 1) / H.bb || hdr != 40u + 4u * (uint32_t)H.nb || hdr > h_in_sizes[i])
            return fail(P, LFC_ERR_CORRUPT, "bad block table");
        if (H.nb > P->block_cap) return fail(P, LFC_ERR_INVALID_ARG, "container has more blocks than the plan holds");
        if ((H.id & 0x80) && (!h_prev || !h_prev[i])) return fail(P, LFC_ERR_INVALID_ARG, "temporal container needs prev");
        if ((uint64_t)nbytes > h_out_bytes[i]) return fail(P, LFC_ERR_CAPACITY, "output frame buffer too small");
        H.sizes.resize(H.nb);
        CK(cudaMemcpyAsync(H.sizes.data(), h_in[i] + 40, 4 * (size_t)H.nb, cudaMemcpyDeviceToHost, P->stream));
        CK(cudaStreamSynchronize(P->stream));
        uint64_t total = hdr;
        for (uint32_t v : H.sizes) total += v;
        if (total != h_in_sizes[i]) return fail(P, LFC_ERR_CORRUPT, "block sizes do not add up to the container");
    }
    int32_t *d_status = ws.mtfreclen;  // block_cap * kTilesPerBlock int32, free while decoding
    int f0 = 0;
    while (f0 < n) {
        std::vector<DecBlockHost> blocks;
        int f1 = f0;
        while (f1 < n && (int)blocks.size() + hd[f1].nb <= P->block_cap) {
            const Hdr &H = hd[f1];
            const int64_t nbytes = 2LL * H.W * H.H;
            uint64_t off = 40 + 4ull * H.nb;
            for (int k = 0; k < H.nb; k++) {
                DecBlockHost d;
                d.src = h_in[f1] + off;
                d.src_len = H.sizes[k];
                d.dst = ws.stream + (size_t)(f1 - f0) * ws.stream_slot + (size_t)k * H.bb;
                d.expect = (int32_t)std::min<int64_t>(H.bb, nbytes - (int64_t)k * H.bb);
                d.pad = 0;
                blocks.push_back(d);
                off += H.sizes[k];
            }
            f1++;
        }
        if (f1 - f0 > P->cfg.max_frames) return fail(P, LFC_ERR_INVALID_ARG, "too many frames");
        const int nb = (int)blocks.size();
        CK(cudaMemcpyAsync(ws.chunk_desc, blocks.data(), sizeof(DecBlockHost) * nb, cudaMemcpyHostToDevice, P->stream));
        CK(launch_bzip2_decode(P, ws.chunk_desc, nb, d_status));
        std::vector<int32_t> st(nb);
        CK(cudaMemcpyAsync(st.data(), d_status, 4 * (size_t)nb, cudaMemcpyDeviceToHost, P->stream));
        CK(cudaStreamSynchronize(P->stream));
        for (int k = 0; k < nb; k++)
            if (st[k] != 0) return fail(P, LFC_ERR_CORRUPT, "bzip2 block failed to decode (code " + std::to_string(st[k]) + ")");
        std::vector<const uint8_t *> outp;
        std::vector<int64_t> outl;
        for (int i = f0; i < f1; i++) {
            const Hdr &H = hd[i];
            const uint16_t *Z = reinterpret_cast<const uint16_t *>(ws.stream + (size_t)(i - f0) * ws.stream_slot);
            const uint16_t *pv = (H.id & 0x80) ? h_prev[i] : nullptr;
            CK(launch_inverse_predict(P, Z, pv, h_out[i], ws.rank, H.W, H.H, H.p, H.id));
            outp.push_back(reinterpret_cast<const uint8_t *>(h_out[i]));
            outl.push_back(2LL * H.W * H.H);
        }
        CK(launch_range_crc(P, outp.data(), outl.data(), f1 - f0, ws.frame_crc));
        std::vector<uint32_t> crc(f1 - f0);
        CK(cudaMemcpyAsync(crc.data(), ws.frame_crc, 4 * (size_t)(f1 - f0), cudaMemcpyDeviceToHost, P->stream));
        CK(cudaStreamSynchronize(P->stream));
        for (int i = f0; i < f1; i++)
            if (crc[i - f0] != hd[i].crc) return fail(P, LFC_ERR_CORRUPT, "frame CRC mismatch");
        f0 = f1;
    }
    return LFC_OK;
}

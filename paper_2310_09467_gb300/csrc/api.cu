// api.cu -- the C ABI of liblfc (include/lfc.h): plans, workspace, and the
// order of the stages (Fig. 1c: prediction, entropy criterion, block bzip2
// coding, header packing). All compute runs in the kernels of this library.
#include "lfc_common.cuh"

#include <algorithm>
#include <cstring>
#include <new>

using namespace lfc;

namespace {

constexpr int kJudgeFramesCap = 16;
constexpr int kDefaultWaitMs = 1000;  // bounded device waits give up after this long

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
    if (id < 0 || id > 255) return false;
    const int f = id_f(id), dom = id_dom(id);
    return dom <= 2 && !(f == 0 && dom != 0);
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
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(P->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
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

extern "C" int lfc_plan_set_tuning(lfc_plan P, const lfc_tuning *t) {
    if (!P || !t) return LFC_ERR_INVALID_ARG;
    lfc_tuning v = P->tune;
    if (t->emit_tile_lenslets) {
        if (t->emit_tile_lenslets != 4 && t->emit_tile_lenslets != 8 && t->emit_tile_lenslets != 16)
            return fail(P, LFC_ERR_INVALID_ARG, "emit_tile_lenslets must be 4, 8 or 16");
        v.emit_tile_lenslets = t->emit_tile_lenslets;
    }
    if (t->chain_range_bytes) {
        const int r = t->chain_range_bytes;
        if (r != 16384 && r != 32768 && r != 65536 && r != 131072 && r != 262144)
            return fail(P, LFC_ERR_INVALID_ARG, "chain_range_bytes must be 16384, 32768, 65536, 131072 or 262144");
        v.chain_range_bytes = t->chain_range_bytes;
    }
    if (t->judge_frames_per_launch) {
        if (t->judge_frames_per_launch < 1 || t->judge_frames_per_launch > P->judge_frames_cap)
            return fail(P, LFC_ERR_INVALID_ARG, "judge_frames_per_launch outside 1..min(max_frames, 16)");
        v.judge_frames_per_launch = t->judge_frames_per_launch;
    }
    if (t->wait_budget_ms) {
        if (t->wait_budget_ms < 1 || t->wait_budget_ms > 60000)
            return fail(P, LFC_ERR_INVALID_ARG, "wait_budget_ms outside 1..60000");
        v.wait_budget_ms = t->wait_budget_ms;
    }
    P->tune = v;
    P->wait_cycles = (long long)(v.wait_budget_ms ? v.wait_budget_ms : kDefaultWaitMs) * P->sm_clock_khz;
    return LFC_OK;
}

extern "C" int lfc_plan_get_tuning(lfc_plan P, lfc_tuning *t) {
    if (!P || !t) return LFC_ERR_INVALID_ARG;
    *t = P->tune;
    if (t->judge_frames_per_launch == 0) t->judge_frames_per_launch = P->judge_frames_cap;
    if (t->wait_budget_ms == 0) t->wait_budget_ms = kDefaultWaitMs;
    return LFC_OK;
}

extern "C" int lfc_plan_bwt_counters(lfc_plan P, int64_t *out, int n) {
    if (!P || !out || n < 0) return 0;
    int k = 0;
    const int64_t head[3] = {P->bwt_calls, P->bwt_rounds, P->bwt_tied_total};
    if (k < n) out[k++] = head[0];
    if (k < n) out[k++] = head[1];
    if (k < n) out[k++] = P->bwt_elements_in;
    if (k < n) out[k++] = head[2];
    for (int r = 0; r < 32 && k < n; r++) out[k++] = P->bwt_round_tied[r];
    return k;
}

extern "C" int lfc_plan_inject_fault(lfc_plan P, int fault) {
    if (!P || fault < 0 || fault > LFC_FAULT_SORT_WITHHOLD) return LFC_ERR_INVALID_ARG;
    // the device word is read by the next suffix sort that runs on the GPU
    // (a call's or a replayed batch's); the withholding tile clears it
    CK(cudaMemsetAsync(P->ws.act_total + kSortFaultWord, fault ? 1 : 0, sizeof(int32_t), P->stream));
    return LFC_OK;
}

extern "C" int lfc_plan_device_status(lfc_plan P) {
    if (!P) return LFC_ERR_INVALID_ARG;
    int32_t st = 0;
    CK(cudaMemcpyAsync(&st, P->ws.act_total + kSortStickyWord, sizeof(int32_t), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    if (st == 0) return LFC_OK;
    CK(cudaMemsetAsync(P->ws.act_total + kSortStickyWord, 0, sizeof(int32_t), P->stream));
    CK(cudaStreamSynchronize(P->stream));
    return st == LFC_ERR_TIMEOUT ? fail(P, LFC_ERR_TIMEOUT, "a bounded device wait gave up") : fail(P, LFC_ERR_CUDA, "device status");
}

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
    void *ptrs[] = {w.hist, w.summ, w.chain_first, w.scores, w.choice, w.jframes, w.cand, w.l2tab, w.stream, w.blocks, w.bstate,
                    w.rle, w.sa, w.sa2, w.rank, w.act, w.act2, w.val, w.val2, w.keys, w.keys2, w.lbstat, w.dhist, w.segbig, w.tileaux, w.bwt,
                    w.mtfidx, w.mtflists, w.mtfrec, w.mtfreclen, w.sym, w.freq, w.rfreq, w.sel, w.lens, w.codes, w.packed, w.cstream, w.masks, w.class_ids,
                    w.act_total, w.block_dst, w.frame_crc, w.crc_part, w.crc_part2, w.chunk_desc, w.dec_tt,
                    w.hx_frames, w.hx_prev, w.hx_out, w.hx_choice, w.hx_sizes};
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
    if (cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, P->device) != cudaSuccess || P->sm_count <= 0)
        P->sm_count = 1;
    if (cudaDeviceGetAttribute(&P->sm_clock_khz, cudaDevAttrClockRate, P->device) != cudaSuccess || P->sm_clock_khz <= 0)
        P->sm_clock_khz = 2100000;
    P->wait_cycles = (long long)kDefaultWaitMs * P->sm_clock_khz;
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
    const int64_t seg_min = chain_seg_bytes(16384);  // smallest tunable segment
    const int64_t segs_max = (n_max + seg_min - 1) / seg_min;
    ws.summ_cap = (int64_t)JF * K * segs_max;
    ws.cstream_kmax = K;
    ws.cstream_slot = (n_max + 255) & ~(int64_t)255;
    ws.stream_slot = (n_max + 255) & ~(int64_t)255;
    ws.stream_words = (stream_bound(bb) + 3) / 4 + 4;
    ws.crc_part_cap = 262144;
    ws.chunk_desc_bytes = 8u << 20;
    cudaError_t e = cudaSuccess;
#define AL(ptr, count)                                           \
    if (e == cudaSuccess) e = dalloc(&ws.ptr, (size_t)(count));
    AL(hist, (size_t)JF * K * kHistBins);
    AL(summ, (size_t)ws.summ_cap * 512);
    AL(scores, (size_t)F * 256);
    AL(choice, (size_t)F);
    AL(jframes, (size_t)JF);
    AL(cand, (size_t)1 << 20);
    AL(l2tab, (size_t)kHistBins);
    AL(stream, (size_t)F * ws.stream_slot);
    AL(cstream, (size_t)JF * K * ws.cstream_slot);
    AL(masks, (size_t)F * 4);
    AL(class_ids, (size_t)64);
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
    AL(keys, (size_t)BC * kBlockCap);
    AL(keys2, (size_t)BC * kBlockCap);
    ws.lbstat_words = (size_t)BC * kTilesPerBlock * 256;
    AL(lbstat, 2 * ws.lbstat_words);
    AL(dhist, (size_t)BC * 8 * 256);
    AL(segbig, (size_t)BC);
    AL(tileaux, (size_t)BC * kTilesPerBlock * 4);
    AL(bwt, (size_t)BC * kBlockCap);
    AL(mtfidx, (size_t)BC * kBlockCap);
    AL(mtflists, (size_t)BC * kTilesPerBlock * 256);
    AL(mtfrec, (size_t)BC * kTilesPerBlock * 256);
    AL(mtfreclen, (size_t)BC * kTilesPerBlock);
    AL(sym, (size_t)BC * (kBlockCap + 64));
    AL(freq, (size_t)BC * kMaxAlpha);
    AL(rfreq, (size_t)BC * kMaxGroups * kMaxAlpha);
    AL(sel, (size_t)BC * kMaxSelectors);
    AL(lens, (size_t)BC * kMaxGroups * kMaxAlpha);
    AL(codes, (size_t)BC * kMaxGroups * kMaxAlpha);
    AL(packed, (size_t)BC * ws.stream_words);
    AL(act_total, (size_t)kSortCtlHead + BC + 1);
    AL(block_dst, (size_t)BC);
    AL(frame_crc, (size_t)F);
    AL(crc_part, (size_t)ws.crc_part_cap);
    AL(crc_part2, (size_t)ws.crc_part_cap);
#undef AL
    // The chain kernel's first-predecessor scratch has one slot per SM, which
    // its shared-memory footprint makes exclusive (no two CTAs fit an SM).
    int smem_sm = 0;
    if (e == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, P->device) == cudaSuccess &&
        2 * chain_smem_bytes() <= (size_t)smem_sm)
        e = cudaErrorNotSupported;
    if (e == cudaSuccess) e = query_nsmid(P->stream, &ws.chain_nsm);
    if (e == cudaSuccess && ws.chain_nsm <= 0) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = dalloc(&ws.chain_first, chain_first_bytes(ws.chain_nsm));
    if (e == cudaSuccess) e = cudaMalloc(&ws.chunk_desc, ws.chunk_desc_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&ws.h_act_total), kSortCtlHead * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.act_total, 0, ((size_t)kSortCtlHead + BC + 1) * sizeof(int32_t), P->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->aux_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->side_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->side_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->side_join, cudaEventDisableTiming);
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
    if (P->aux_stream) cudaStreamDestroy(P->aux_stream);
    if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
    if (P->side_stream) cudaStreamDestroy(P->side_stream);
    if (P->side_fork) cudaEventDestroy(P->side_fork);
    if (P->side_join) cudaEventDestroy(P->side_join);
    delete P;
}

// ------------------------------------------------------- descriptor arena
// Every call first lays out all of its descriptor tables on the host, copies
// them to the device once, then only launches kernels. A batch keeps its
// arena and replays the launches as a CUDA graph.
namespace {

struct Arena {
    std::vector<uint8_t> host;
    size_t reserve(size_t n) {
        const size_t o = (host.size() + 15) & ~(size_t)15;
        host.resize(o + n);
        return o;
    }
    size_t put(const void *p, size_t n) {
        const size_t o = reserve(n);
        if (n) memcpy(host.data() + o, p, n);
        return o;
    }
};

struct JudgeChunk {
    size_t off_tables = 0, off_cand = 0;
    int nf = 0;
    int64_t ctas = 0, nhist = 0;
    JudgeLaunch L{};
};

struct CoderPass {
    size_t off_blocks = 0, off_crc = 0, off_fo = 0;
    int nblocks = 0, max_m = 0, f0 = 0, f1 = 0;
    CrcRun crc;
    std::vector<BlockDesc> blocks;
};

struct CompressDesc {
    std::vector<lfc_frame> frames;
    Arena arena;
    std::vector<JudgeChunk> judge;
    CrcRun frame_crc;
    size_t off_frame_crc = 0, off_dst = 0;
    std::vector<CoderPass> passes;
    std::vector<FrameDev> fd;
    std::vector<uint8_t *> dst;
    int n = 0, bb = 0;
};

bool capturing(lfc_plan P) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(P->stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone;
}

// Bytes a chain warp walks in one launch: at most the tuned range, chosen so
// that the launch's CTAs fill whole waves of one CTA per SM. A candidate
// range r gives sum_f K_f ceil(n_f / seg(r)) CTAs; its cost is taken as the
// waves those need times (r + a fixed per-CTA share of 8 KB). Candidates: the
// equal splits of the largest stream into s >= s0 segments (s0 the count at
// the tuned range), at most 2 s0, a multiple of 512 bytes, >= 16 KB.
int chain_range_for(lfc_plan P, const lfc_frame *frames, int nf) {
    const int tuned = P->tune.chain_range_bytes;
    int64_t n_max = 0;
    int k_spatial = (int)P->ids_spatial.size(), k_all = k_spatial + (int)P->ids_temporal.size();
    for (int i = 0; i < nf; i++) n_max = std::max<int64_t>(n_max, 2LL * frames[i].width * frames[i].height);
    if (n_max <= 0) return tuned;
    const int64_t w = chain_seg_bytes(1);  // warps per CTA
    const int64_t s0 = std::max<int64_t>(1, (n_max + w * tuned - 1) / (w * tuned));
    int best = tuned;
    double best_cost = -1.0;
    for (int64_t s = s0; s <= 2 * s0; s++) {
        int64_t r = (n_max + w * s - 1) / (w * s);
        r = (r + 511) / 512 * 512;
        if (r > tuned || r < 16384) continue;
        int64_t ctas = 0;
        for (int i = 0; i < nf; i++) {
            const int64_t nb = 2LL * frames[i].width * frames[i].height;
            const int K = (frames[i].prev != nullptr && !P->ids_temporal.empty()) ? k_all : k_spatial;
            ctas += (int64_t)K * ((nb + w * r - 1) / (w * r));
        }
        const int64_t waves = (ctas + P->sm_count - 1) / P->sm_count;
        const double cost = (double)waves * (double)(r + 8192);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = (int)r;
        }
    }
    return best;
}

int build_judge(lfc_plan P, const lfc_frame *frames, int n, Arena &A, std::vector<JudgeChunk> &out) {
    Workspace &ws = P->ws;
    const int per_launch = P->tune.judge_frames_per_launch > 0 ? P->tune.judge_frames_per_launch : P->judge_frames_cap;
    for (int f0 = 0; f0 < n; f0 += per_launch) {
        const int f1 = std::min(n, f0 + per_launch);
        const int nf = f1 - f0;
        const int range = chain_range_for(P, frames + f0, nf);
        const int64_t seg_bytes = chain_seg_bytes(range);
        std::vector<JudgeFrame> jf(nf);
        std::vector<int32_t> frame_index(nf), hist_frame;
        std::vector<uint8_t> cand;
        int64_t cta = 0, hist = 0, summ = 0;
        JudgeChunk C;
        C.L = JudgeLaunch{0, 16, 0, 0, 0, range};
        for (int i = 0; i < nf; i++) {
            const lfc_frame &fr = frames[f0 + i];
            const bool tmp = fr.prev != nullptr && !P->ids_temporal.empty();
            JudgeFrame &J = jf[i];
            J.F = to_dev(fr, tmp);
            J.cand_off = (int32_t)cand.size();
            uint32_t fset[2] = {0, 0}, fall[2] = {0, 0};  // f with a residual field / with any candidate
            for (uint8_t id : P->ids_spatial) cand.push_back(id);
            if (tmp)
                for (uint8_t id : P->ids_temporal) cand.push_back(id);
            for (size_t k = J.cand_off; k < cand.size(); k++) {
                const int id = cand[k], f = id_f(id), dom = id_dom(id);
                if (f && dom != 1) fset[(id >> 7) & 1] |= 1u << f;
                if (f) fall[(id >> 7) & 1] |= 1u << f;
            }
            // shared-memory slots of the emission kernel: residual fields and symbol planes
            for (int kd = 0; kd < 2; kd++)
                C.L.nslots_max = std::max(C.L.nslots_max,
                                          std::max(__builtin_popcount(fset[kd]), __builtin_popcount(fall[kd])));
            C.L.any_temporal |= tmp ? 1 : 0;
            C.L.max_p = std::max(C.L.max_p, fr.pitch);
            J.K = (int32_t)(cand.size() - J.cand_off);
            const int64_t nbytes = 2LL * fr.width * fr.height;
            J.rows_per_seg = 0;
            J.segs = (int32_t)((nbytes + seg_bytes - 1) / seg_bytes);
            J.cta_base = cta;
            J.hist_off = hist;
            J.summ_off = summ;
            J.mask = (P->cnn && P->topk > 0 && !tmp) ? ws.masks + (size_t)4 * (f0 + i) : nullptr;
            cta += (int64_t)J.K * J.segs;
            summ += (int64_t)J.K * J.segs;
            for (int k = 0; k < J.K; k++) hist_frame.push_back(i);
            hist += J.K;
            frame_index[i] = f0 + i;
        }
        // lenslets per emission tile: the tuned width, narrowed until it fits
        C.L.TS = P->tune.emit_tile_lenslets;
        while (C.L.TS > 1 && emit_all_smem_bytes(C.L.max_p, C.L.TS, C.L.nslots_max) > 200 * 1024) C.L.TS /= 2;
        if (emit_all_smem_bytes(C.L.max_p, C.L.TS, C.L.nslots_max) > 200 * 1024)
            return fail(P, LFC_ERR_INVALID_ARG, "pitch too large for the emission tile");
        for (int i = 0; i < nf; i++) {
            const FrameDev &F = jf[i].F;
            C.L.max_tiles = std::max(C.L.max_tiles, F.Ny * ((F.Nx + C.L.TS - 1) / C.L.TS));
        }
        if (summ > ws.summ_cap) return fail(P, LFC_ERR_INVALID_ARG, "judge summary capacity exceeded");
        // frames | frame_index | hist_frame (the kernels find the tables behind the frames)
        std::vector<uint8_t> t(sizeof(JudgeFrame) * nf + 4 * nf + 4 * hist_frame.size());
        memcpy(t.data(), jf.data(), sizeof(JudgeFrame) * nf);
        memcpy(t.data() + sizeof(JudgeFrame) * nf, frame_index.data(), 4 * nf);
        memcpy(t.data() + sizeof(JudgeFrame) * nf + 4 * nf, hist_frame.data(), 4 * hist_frame.size());
        C.off_tables = A.put(t.data(), t.size());
        C.off_cand = A.put(cand.data(), cand.size());
        C.nf = nf;
        C.ctas = cta;
        C.nhist = hist;
        out.push_back(C);
    }
    return LFC_OK;
}

// d_dst (device array of the frames' stream slots, may be null): the chosen
// stream of each frame is copied out of the judge's candidate streams.
int run_judge(lfc_plan P, const std::vector<lfc_frame> &frames, const std::vector<JudgeChunk> &chunks,
              const uint8_t *d_arena, uint8_t *d_choice, uint64_t *d_scores, uint8_t *const *d_dst = nullptr) {
    if (P->cnn && P->topk > 0) {
        const int r = cnn_propose(P->cnn, frames.data(), (int)frames.size(), P->ws.class_ids, P->topk, P->tau, P->ws.masks,
                                  P->stream);
        if (r) return fail(P, r, "proposal network failed");
    }
    int f0 = 0;
    for (const JudgeChunk &C : chunks) {
        CK(launch_judge(P, reinterpret_cast<const JudgeFrame *>(d_arena + C.off_tables), C.nf, C.ctas, C.L,
                        d_arena + C.off_cand, C.nhist, d_scores, d_choice));
        if (d_dst) {
            stage_begin(P, LFC_STAGE_EMIT);
            CK(launch_copy_chosen(P, reinterpret_cast<const JudgeFrame *>(d_arena + C.off_tables), C.nf,
                                  d_arena + C.off_cand, d_choice, d_dst));
            stage_end(P, LFC_STAGE_EMIT);
        }
        f0 += C.nf;
    }
    return LFC_OK;
}

// Coder descriptors for one pass over the given blocks.
void build_pass(Arena &A, CoderPass &cp) {
    int max_len = 0;
    std::vector<const uint8_t *> ptr(cp.blocks.size());
    std::vector<int64_t> len(cp.blocks.size());
    for (size_t b = 0; b < cp.blocks.size(); b++) {
        max_len = std::max(max_len, cp.blocks[b].len);
        ptr[b] = cp.blocks[b].src;
        len[b] = cp.blocks[b].len;
    }
    cp.nblocks = (int)cp.blocks.size();
    cp.max_m = std::min(kRleCap, max_len + max_len / 4 + 4);
    cp.off_blocks = A.put(cp.blocks.data(), sizeof(BlockDesc) * cp.blocks.size());
    const int nchunks = crc_count_chunks(len.data(), cp.nblocks);
    cp.off_crc = A.reserve(crc_table_bytes(nchunks, cp.nblocks));
    crc_build_tables(ptr.data(), len.data(), cp.nblocks, A.host.data() + cp.off_crc, &cp.crc);
}

int run_pass(lfc_plan P, const CoderPass &cp, const uint8_t *d_arena) {
    Workspace &ws = P->ws;
    const int nb = cp.nblocks;
    for (const BlockDesc &b : cp.blocks) P->bwt_elements_in += b.len;
    CK(cudaMemsetAsync(ws.bstate, 0, sizeof(BlockState) * nb, P->stream));
    // block CRCs on the side stream, overlapped with RLE1 and the BWT (each
    // writes only its own word of the block state; packing reads it)
    CK(cudaEventRecord(P->side_fork, P->stream));
    CK(cudaStreamWaitEvent(P->side_stream, P->side_fork, 0));
    CK(launch_crc(P, d_arena + cp.off_crc, cp.crc, &ws.bstate[0].crc, (int)(sizeof(BlockState) / 4), P->side_stream));
    CK(cudaEventRecord(P->side_join, P->side_stream));
    stage_begin(P, LFC_STAGE_RLE1);
    CK(launch_rle1(P, nb, reinterpret_cast<const BlockDesc *>(d_arena + cp.off_blocks)));
    stage_end(P, LFC_STAGE_RLE1);
    P->bwt_timed_out = false;
    CK(launch_bwt(P, nb, cp.max_m));
    if (P->bwt_timed_out) return fail(P, LFC_ERR_TIMEOUT, "suffix sort: a bounded look-back wait gave up");
    stage_begin(P, LFC_STAGE_MTF);
    CK(launch_mtf_rle2(P, nb));
    stage_end(P, LFC_STAGE_MTF);
    stage_begin(P, LFC_STAGE_HUFFMAN);
    CK(launch_huffman(P, nb));
    stage_end(P, LFC_STAGE_HUFFMAN);
    CK(cudaStreamWaitEvent(P->stream, P->side_join, 0));
    stage_begin(P, LFC_STAGE_PACK);
    CK(launch_pack(P, nb));
    stage_end(P, LFC_STAGE_PACK);
    return LFC_OK;
}

int check_frames(lfc_plan P, const lfc_frame *frames, int n) {
    if (!P || !frames || n < 1) return fail(P, LFC_ERR_INVALID_ARG, "bad frame list");
    if (n > P->cfg.max_frames) return fail(P, LFC_ERR_INVALID_ARG, "n > max_frames");
    for (int i = 0; i < n; i++) {
        const int r = check_frame(P, frames[i]);
        if (r) return r;
    }
    return LFC_OK;
}

int build_compress(lfc_plan P, const lfc_frame *frames, int n, bool judge, size_t out_cap, CompressDesc &D,
                   std::vector<uint64_t> &out_off) {
    Workspace &ws = P->ws;
    const int bb = block_bytes_of(P);
    D.n = n;
    D.bb = bb;
    D.frames.assign(frames, frames + n);
    out_off.resize(n);
    uint64_t need = 0;
    for (int i = 0; i < n; i++) {
        out_off[i] = need;
        need += container_bound(frames[i].width, frames[i].height, bb);
    }
    if (need > out_cap) return fail(P, LFC_ERR_CAPACITY, "lfc_compress: out_cap below the sum of container bounds");
    if (judge) {
        const int r = build_judge(P, frames, n, D.arena, D.judge);
        if (r) return r;
    }
    D.fd.resize(n);
    D.dst.resize(n);
    std::vector<const uint8_t *> raw(n);
    std::vector<int64_t> rawlen(n);
    for (int i = 0; i < n; i++) {
        D.fd[i] = to_dev(frames[i], frames[i].prev != nullptr);
        D.dst[i] = ws.stream + (size_t)i * ws.stream_slot;
        raw[i] = reinterpret_cast<const uint8_t *>(frames[i].data);
        rawlen[i] = 2LL * frames[i].width * frames[i].height;
    }
    D.off_dst = D.arena.put(D.dst.data(), sizeof(uint8_t *) * (size_t)n);
    const int nck = crc_count_chunks(rawlen.data(), n);
    D.off_frame_crc = D.arena.reserve(crc_table_bytes(nck, n));
    crc_build_tables(raw.data(), rawlen.data(), n, D.arena.host.data() + D.off_frame_crc, &D.frame_crc);
    int f0 = 0;
    while (f0 < n) {
        CoderPass cp;
        std::vector<FrameOut> fo;
        int f1 = f0;
        while (f1 < n) {
            const int64_t nbytes = rawlen[f1];
            const int64_t nbf = (nbytes + bb - 1) / bb;
            if ((int64_t)cp.blocks.size() + nbf > P->block_cap) break;
            FrameOut F;
            F.out_off = out_off[f1];
            F.block0 = (int32_t)cp.blocks.size();
            F.nblocks = (int32_t)nbf;
            F.W = frames[f1].width;
            F.H = frames[f1].height;
            F.p = frames[f1].pitch;
            F.pad = 0;
            fo.push_back(F);
            for (int64_t k = 0; k < nbf; k++) {
                BlockDesc d;
                d.src = D.dst[f1] + k * bb;
                d.len = (int32_t)std::min<int64_t>(bb, nbytes - k * bb);
                d.frame = f1;
                cp.blocks.push_back(d);
            }
            f1++;
        }
        if (f1 == f0) return fail(P, LFC_ERR_INVALID_ARG, "lfc_compress: frame needs more blocks than the plan holds");
        cp.f0 = f0;
        cp.f1 = f1;
        build_pass(D.arena, cp);
        cp.off_fo = D.arena.put(fo.data(), sizeof(FrameOut) * fo.size());
        D.passes.push_back(std::move(cp));
        f0 = f1;
    }
    return LFC_OK;
}

int run_compress(lfc_plan P, const CompressDesc &D, const uint8_t *d_arena, const uint8_t *d_choice, uint8_t *d_out,
                 uint64_t *d_out_sizes) {
    Workspace &ws = P->ws;
    const uint8_t *choice = d_choice;
    // frame CRCs of the raw frames do not depend on the judge: side stream
    CK(cudaEventRecord(P->side_fork, P->stream));
    CK(cudaStreamWaitEvent(P->side_stream, P->side_fork, 0));
    CK(launch_crc(P, d_arena + D.off_frame_crc, D.frame_crc, ws.frame_crc, 1, P->side_stream, ws.crc_part2));
    CK(cudaEventRecord(P->side_join, P->side_stream));
    if (!D.judge.empty()) {  // the judge also copies out the chosen streams
        const int r = run_judge(P, D.frames, D.judge, d_arena, ws.choice, ws.scores,
                                reinterpret_cast<uint8_t *const *>(d_arena + D.off_dst));
        if (r) return r;
        choice = ws.choice;
    } else {
        stage_begin(P, LFC_STAGE_EMIT);
        CK(launch_emit(D.fd.data(), choice, D.n, D.dst.data(), P->stream));
        count_launches(P, (D.n + 7) / 8);
        stage_end(P, LFC_STAGE_EMIT);
    }
    CK(cudaStreamWaitEvent(P->stream, P->side_join, 0));
    for (const CoderPass &cp : D.passes) {
        const int r = run_pass(P, cp, d_arena);
        if (r) return r;
        stage_begin(P, LFC_STAGE_CONTAINER);
        CK(launch_container(P, cp.f1 - cp.f0, cp.nblocks, reinterpret_cast<const FrameOut *>(d_arena + cp.off_fo),
                            choice + cp.f0, ws.frame_crc + cp.f0, d_out, d_out_sizes + cp.f0, D.bb));
        stage_end(P, LFC_STAGE_CONTAINER);
    }
    return LFC_OK;
}

int stage_arena(lfc_plan P, const Arena &A) {
    if (A.host.size() > P->ws.chunk_desc_bytes) return fail(P, LFC_ERR_INVALID_ARG, "descriptor tables exceed the plan's staging buffer");
    if (!A.host.empty())
        CK(cudaMemcpyAsync(P->ws.chunk_desc, A.host.data(), A.host.size(), cudaMemcpyHostToDevice, P->stream));
    return LFC_OK;
}

}  // namespace

extern "C" int lfc_judge(lfc_plan P, const lfc_frame *frames, int n, uint8_t *d_choice, uint64_t *d_scores) {
    if (!P || !d_choice) return fail(P, LFC_ERR_INVALID_ARG, "lfc_judge: bad arguments");
    int r = check_frames(P, frames, n);
    if (r) return r;
    Arena A;
    std::vector<JudgeChunk> chunks;
    r = build_judge(P, frames, n, A, chunks);
    if (r) return r;
    r = stage_arena(P, A);
    if (r) return r;
    return run_judge(P, std::vector<lfc_frame>(frames, frames + n), chunks, reinterpret_cast<const uint8_t *>(P->ws.chunk_desc),
                     d_choice, d_scores ? d_scores : P->ws.scores);
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

extern "C" int lfc_bzip2_encode(lfc_plan P, const uint8_t *d_in, const uint64_t *h_offsets, const uint32_t *h_sizes,
                                int n_blocks, uint8_t *d_out, size_t out_stride, uint32_t *d_stream_sizes) {
    if (!P || !d_in || !h_offsets || !h_sizes || !d_out || !d_stream_sizes || n_blocks < 1)
        return fail(P, LFC_ERR_INVALID_ARG, "lfc_bzip2_encode: bad arguments");
    if (n_blocks > P->block_cap) return fail(P, LFC_ERR_INVALID_ARG, "lfc_bzip2_encode: too many blocks");
    CoderPass cp;
    uint32_t max_size = 0;
    for (int b = 0; b < n_blocks; b++) {
        if (h_sizes[b] < 1 || h_sizes[b] > (uint32_t)kMaxBlockBytes)
            return fail(P, LFC_ERR_INVALID_ARG, "lfc_bzip2_encode: block size outside 1..720000");
        BlockDesc d;
        d.src = d_in + h_offsets[b];
        d.len = (int32_t)h_sizes[b];
        d.frame = -1;
        cp.blocks.push_back(d);
        max_size = std::max(max_size, h_sizes[b]);
    }
    if (out_stride < (size_t)stream_bound(max_size)) return fail(P, LFC_ERR_CAPACITY, "lfc_bzip2_encode: out_stride too small");
    Arena A;
    build_pass(A, cp);
    int r = stage_arena(P, A);
    if (r) return r;
    r = run_pass(P, cp, reinterpret_cast<const uint8_t *>(P->ws.chunk_desc));
    if (r) return r;
    stage_begin(P, LFC_STAGE_CONTAINER);
    CK(launch_copy_streams(P, n_blocks, d_out, out_stride, d_stream_sizes));
    stage_end(P, LFC_STAGE_CONTAINER);
    return LFC_OK;
}

extern "C" int lfc_bwt_blocks(lfc_plan P, const uint8_t *d_in, const uint64_t *h_offsets, const uint32_t *h_sizes,
                              int n_blocks, uint8_t *d_L, size_t L_stride, uint32_t *d_len, uint32_t *d_orig) {
    if (!P || !d_in || !h_offsets || !h_sizes || !d_L || !d_len || !d_orig || n_blocks < 1)
        return fail(P, LFC_ERR_INVALID_ARG, "lfc_bwt_blocks: bad arguments");
    if (n_blocks > P->block_cap) return fail(P, LFC_ERR_INVALID_ARG, "lfc_bwt_blocks: too many blocks");
    CoderPass cp;
    uint32_t max_size = 0;
    for (int b = 0; b < n_blocks; b++) {
        if (h_sizes[b] < 1 || h_sizes[b] > (uint32_t)kMaxBlockBytes)
            return fail(P, LFC_ERR_INVALID_ARG, "lfc_bwt_blocks: block size outside 1..720000");
        BlockDesc d;
        d.src = d_in + h_offsets[b];
        d.len = (int32_t)h_sizes[b];
        d.frame = -1;
        cp.blocks.push_back(d);
        max_size = std::max(max_size, h_sizes[b]);
    }
    const size_t need = std::min<size_t>((size_t)kRleCap, (size_t)max_size + max_size / 4 + 4);
    if (L_stride < need) return fail(P, LFC_ERR_CAPACITY, "lfc_bwt_blocks: L_stride below the RLE1 bound");
    Arena A;
    build_pass(A, cp);
    int r = stage_arena(P, A);
    if (r) return r;
    const BlockDesc *d_blocks = reinterpret_cast<const BlockDesc *>(reinterpret_cast<const uint8_t *>(P->ws.chunk_desc) + cp.off_blocks);
    CK(cudaMemsetAsync(P->ws.bstate, 0, sizeof(BlockState) * cp.nblocks, P->stream));
    CK(launch_rle1(P, cp.nblocks, d_blocks));
    P->bwt_timed_out = false;
    CK(launch_bwt(P, cp.nblocks, cp.max_m));
    if (P->bwt_timed_out) return fail(P, LFC_ERR_TIMEOUT, "suffix sort: a bounded look-back wait gave up");
    CK(launch_copy_bwt(P, cp.nblocks, d_L, L_stride, d_len, d_orig));
    return LFC_OK;
}

extern "C" int lfc_compress(lfc_plan P, const lfc_frame *frames, int n, const uint8_t *d_choice, uint8_t *d_out,
                            size_t out_cap, uint64_t *d_out_sizes) {
    if (!P || !d_out || !d_out_sizes) return fail(P, LFC_ERR_INVALID_ARG, "lfc_compress: bad arguments");
    int r = check_frames(P, frames, n);
    if (r) return r;
    CompressDesc D;
    std::vector<uint64_t> out_off;
    r = build_compress(P, frames, n, d_choice == nullptr, out_cap, D, out_off);
    if (r) return r;
    r = stage_arena(P, D.arena);
    if (r) return r;
    return run_compress(P, D, reinterpret_cast<const uint8_t *>(P->ws.chunk_desc), d_choice, d_out, d_out_sizes);
}

extern "C" int lfc_compress_host(lfc_plan P, const lfc_frame *h_frames, int n, const uint8_t *h_choice, uint8_t *h_out,
                                 size_t out_cap, uint64_t *h_out_sizes) {
    if (!P || !h_frames || !h_out || !h_out_sizes || n < 1)
        return fail(P, LFC_ERR_INVALID_ARG, "lfc_compress_host: bad arguments");
    if (n > P->cfg.max_frames) return fail(P, LFC_ERR_INVALID_ARG, "lfc_compress_host: n > max_frames");
    Workspace &ws = P->ws;
    const int bb = block_bytes_of(P);
    const size_t slot = 2 * (size_t)P->cfg.width * P->cfg.height;
    // the containers' slots in h_out, as lfc_compress lays them out
    std::vector<uint64_t> off(n);
    uint64_t need = 0;
    bool any_prev = false;
    for (int i = 0; i < n; i++) {
        const int r = check_frame(P, h_frames[i]);
        if (r) return r;
        off[i] = need;
        need += container_bound(h_frames[i].width, h_frames[i].height, bb);
        any_prev |= h_frames[i].prev != nullptr;
    }
    if (need > out_cap) return fail(P, LFC_ERR_CAPACITY, "lfc_compress_host: out_cap below the sum of container bounds");
    // staging for the plan's largest call, allocated once
    const int F = P->cfg.max_frames;
    const size_t out_all = (size_t)F * container_bound(P->cfg.width, P->cfg.height, bb);
    cudaError_t e = cudaSuccess;
    if (!ws.hx_frames) e = cudaMalloc(reinterpret_cast<void **>(&ws.hx_frames), (size_t)F * slot);
    if (e == cudaSuccess && any_prev && !ws.hx_prev) e = cudaMalloc(reinterpret_cast<void **>(&ws.hx_prev), (size_t)F * slot);
    if (e == cudaSuccess && !ws.hx_out) {
        e = cudaMalloc(reinterpret_cast<void **>(&ws.hx_out), out_all);
        ws.hx_out_cap = out_all;
    }
    if (e == cudaSuccess && !ws.hx_sizes) e = cudaMalloc(reinterpret_cast<void **>(&ws.hx_sizes), (size_t)F * sizeof(uint64_t));
    if (e == cudaSuccess && !ws.hx_choice) e = cudaMalloc(reinterpret_cast<void **>(&ws.hx_choice), (size_t)F);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(P, LFC_ERR_NOMEM, "lfc_compress_host: staging allocation", e);
    }
    // frames in, one copy each (pinned host memory makes them asynchronous)
    std::vector<lfc_frame> dev(h_frames, h_frames + n);
    for (int i = 0; i < n; i++) {
        const size_t bytes = 2 * (size_t)h_frames[i].width * h_frames[i].height;
        dev[i].data = reinterpret_cast<const uint16_t *>(ws.hx_frames + (size_t)i * slot);
        CK(cudaMemcpyAsync(ws.hx_frames + (size_t)i * slot, h_frames[i].data, bytes, cudaMemcpyHostToDevice, P->stream));
        if (h_frames[i].prev) {
            dev[i].prev = reinterpret_cast<const uint16_t *>(ws.hx_prev + (size_t)i * slot);
            CK(cudaMemcpyAsync(ws.hx_prev + (size_t)i * slot, h_frames[i].prev, bytes, cudaMemcpyHostToDevice, P->stream));
        }
    }
    if (h_choice) CK(cudaMemcpyAsync(ws.hx_choice, h_choice, (size_t)n, cudaMemcpyHostToDevice, P->stream));
    const int r = lfc_compress(P, dev.data(), n, h_choice ? ws.hx_choice : nullptr, ws.hx_out, ws.hx_out_cap, ws.hx_sizes);
    if (r) return r;
    // sizes, then each container's bytes, out
    CK(cudaMemcpyAsync(h_out_sizes, ws.hx_sizes, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    for (int i = 0; i < n; i++)  // a size beyond its slot would overrun h_out: never copy it
        if (h_out_sizes[i] > container_bound(h_frames[i].width, h_frames[i].height, bb))
            return fail(P, LFC_ERR_CUDA, "lfc_compress_host: container size beyond its slot");
    for (int i = 0; i < n; i++)
        CK(cudaMemcpyAsync(h_out + off[i], ws.hx_out + off[i], (size_t)h_out_sizes[i], cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    return LFC_OK;
}

// ------------------------------------------------------------------ batches
struct lfc_batch_s {
    lfc_plan P = nullptr;
    uint8_t *d_arena = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t nodes = 0;
};

extern "C" int lfc_batch_create(lfc_plan P, const lfc_frame *frames, int n, const uint8_t *d_choice, uint8_t *d_out,
                                size_t out_cap, uint64_t *d_out_sizes, lfc_batch *out) {
    if (!P || !d_out || !d_out_sizes || !out) return fail(P, LFC_ERR_INVALID_ARG, "lfc_batch_create: bad arguments");
    *out = nullptr;
    int r = check_frames(P, frames, n);
    if (r) return r;
    CompressDesc D;
    std::vector<uint64_t> out_off;
    r = build_compress(P, frames, n, d_choice == nullptr, out_cap, D, out_off);
    if (r) return r;
    lfc_batch B = new (std::nothrow) lfc_batch_s();
    if (!B) return fail(P, LFC_ERR_NOMEM, "lfc_batch_create: host allocation");
    B->P = P;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&B->d_arena), std::max<size_t>(D.arena.host.size(), 16));
    if (e == cudaSuccess && !D.arena.host.empty())
        e = cudaMemcpy(B->d_arena, D.arena.host.data(), D.arena.host.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) {
        if (B->d_arena) cudaFree(B->d_arena);
        delete B;
        return fail(P, e == cudaErrorMemoryAllocation ? LFC_ERR_NOMEM : LFC_ERR_CUDA, "lfc_batch_create: arena", e);
    }
    // record on the plan's capture stream (the plan's own stream may be the
    // legacy default stream, which cannot be captured); replay on the plan's
    // stream
    const bool was_timing = P->timing;
    P->timing = false;
    const int64_t l0 = P->launches;
    cudaStream_t home = P->stream;
    P->stream = P->cap_stream;
    e = cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal);
    int rr = e == cudaSuccess ? run_compress(P, D, B->d_arena, d_choice, d_out, d_out_sizes)
                              : fail(P, LFC_ERR_CUDA, "lfc_batch_create: begin capture", e);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(P->stream, &g);
    P->stream = home;
    P->timing = was_timing;
    B->nodes = P->launches - l0;
    P->launches = l0;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && rr == LFC_OK) e = cudaGraphInstantiate(&B->exec, g, 0);
    B->graph = g;
    if (e != cudaSuccess || rr != LFC_OK) {
        if (B->exec) cudaGraphExecDestroy(B->exec);
        if (g) cudaGraphDestroy(g);
        cudaFree(B->d_arena);
        delete B;
        cudaGetLastError();
        return rr != LFC_OK ? rr : fail(P, LFC_ERR_CUDA, "lfc_batch_create: graph capture", e);
    }
    *out = B;
    return LFC_OK;
}

extern "C" int lfc_batch_launch(lfc_batch B) {
    if (!B) return LFC_ERR_INVALID_ARG;
    lfc_plan P = B->P;
    CK(cudaGraphLaunch(B->exec, P->stream));
    P->launches += B->nodes;
    return LFC_OK;
}

extern "C" void lfc_batch_destroy(lfc_batch B) {
    if (!B) return;
    cudaStreamSynchronize(B->P->stream);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->d_arena) cudaFree(B->d_arena);
    delete B;
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
        for (int k = 0; k < nb; k++) {
            if (st[k] != 0) return fail(P, LFC_ERR_CORRUPT, "bzip2 block failed to decode (code " + std::to_string(st[k]) + ")");
        }
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

// ------------------------------------------------------- learned proposal
extern "C" int lfc_plan_set_proposal(lfc_plan P, lfc_cnn cnn, const uint8_t *h_class_ids, int n_classes, int topk,
                                     float tau) {
    if (!P) return LFC_ERR_INVALID_ARG;
    if (!cnn) {
        P->cnn = nullptr;
        P->topk = 0;
        return LFC_OK;
    }
    if (!h_class_ids || n_classes != cnn_classes(cnn) || n_classes > 64 || topk < 1 || topk > n_classes)
        return fail(P, LFC_ERR_INVALID_ARG, "lfc_plan_set_proposal: classes or topk");
    for (int k = 0; k < n_classes; k++)
        if (!id_valid(h_class_ids[k]) || (h_class_ids[k] & 0x80)) return fail(P, LFC_ERR_INVALID_ARG, "lfc_plan_set_proposal: class id");
    CK(cudaMemcpy(P->ws.class_ids, h_class_ids, (size_t)n_classes, cudaMemcpyHostToDevice));
    P->cnn = cnn;
    P->topk = topk;
    P->tau = tau;
    return LFC_OK;
}

extern "C" int lfc_propose(lfc_plan P, const lfc_frame *frames, int n, uint64_t *d_masks) {
    if (!P || !d_masks) return fail(P, LFC_ERR_INVALID_ARG, "lfc_propose: bad arguments");
    if (!P->cnn) return fail(P, LFC_ERR_INVALID_ARG, "lfc_propose: no network attached");
    const int r = check_frames(P, frames, n);
    if (r) return r;
    const int rr = cnn_propose(P->cnn, frames, n, P->ws.class_ids, P->topk, P->tau, d_masks, P->stream);
    return rr ? fail(P, rr, "proposal network failed") : LFC_OK;
}


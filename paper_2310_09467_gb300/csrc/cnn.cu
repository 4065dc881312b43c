// cnn.cu -- learned candidate proposal (the paper motivates reducing the
// criterion's time, Sec. 4): a 4-layer 3x3 convolutional network on a
// 2 x 256 x 256 thumbnail of the frame predicts the judge's choice.
//
// Layout: activations NHWC in BF16 ([frame][y][x][channel], 32 channels;
// the 2-channel input is padded to 16), master parameters FP32.
// Forward and input-gradient convolutions are implicit GEMMs on the tensor
// cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation): one CTA per
// 8 x 16 output tile, one warp per 16-pixel row, the input tile with its
// halo and all 9 x 32 x Cin weights staged in shared memory. Weight
// gradients are FP32 outer products on the CUDA cores over row bands.
#include "lfc_common.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace lfc {

constexpr int kT = 256;   // thumbnail side
constexpr int kCh = 32;   // hidden channels
constexpr int kC0 = 16;   // padded input channels (2 used)
constexpr int kPix = kT * kT;

typedef __nv_bfloat16 bf16;

struct POff {
    size_t w[4], b[4], wl, bl, total;
};

static POff param_offsets(int K) {
    POff o;
    const int cin[4] = {2, kCh, kCh, kCh};
    size_t at = 0;
    for (int l = 0; l < 4; l++) {
        o.w[l] = at;
        at += (size_t)9 * cin[l] * kCh;   // [ky][kx][ci][co]
        o.b[l] = at;
        at += kCh;
    }
    o.wl = at;
    at += (size_t)kCh * K;                // [c][k]
    o.bl = at;
    at += K;
    o.total = at;
    return o;
}

}  // namespace lfc

struct lfc_cnn_s {
    int K = 0, max_batch = 0;
    cudaStream_t stream = nullptr;
    lfc::POff off;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    int64_t step = 0;
    lfc::bf16 *wf[4] = {};   // forward B operand [9][32 co][cin_pad ci]
    lfc::bf16 *wd[4] = {};   // input-gradient B operand [9][32 ci][32 co], flipped taps
    lfc::bf16 *x0 = nullptr; // [B][256][256][16]
    lfc::bf16 *act[4] = {};  // [B][256][256][32]
    lfc::bf16 *dpre[2] = {}; // [B][256][256][32]
    float *gap_part = nullptr, *gap = nullptr, *probs = nullptr, *dz = nullptr, *dg = nullptr, *loss = nullptr;
    std::string err;
};

namespace lfc {

// ------------------------------------------------------------ thumbnails
// channel 0: raw layout, channel 1: view-major mosaic; bs x bs block means
// (edge blocks over their valid pixels), log1p(max(mean - 100, 0)) / 8.
__global__ void thumb_kernel(FrameDev F, int bs, bf16 *__restrict__ x0, float *__restrict__ thumbs) {
    const int tx = blockIdx.x * blockDim.x + threadIdx.x, ty = blockIdx.y;
    if (tx >= kT) return;
    const int th = (F.H + bs - 1) / bs, tw = (F.W + bs - 1) / bs;
    float val[2] = {0.f, 0.f};
    if (ty < th && tx < tw) {
        const int ya = ty * bs, yb = min(F.H, ya + bs), xa = tx * bs, xb = min(F.W, xa + bs);
        float s0 = 0.f, s1 = 0.f;
        for (int y = ya; y < yb; y++) {
            for (int x = xa; x < xb; x++) {
                s0 += (float)__ldg(F.X + (size_t)y * F.W + x);
                // mosaic pixel (y, x) = raw pixel ((y % Ny) p + y / Ny, (x % Nx) p + x / Nx)
                const int ry = (y % F.Ny) * F.p + y / F.Ny, rx = (x % F.Nx) * F.p + x / F.Nx;
                s1 += (float)__ldg(F.X + (size_t)ry * F.W + rx);
            }
        }
        const float cnt = (float)((yb - ya) * (xb - xa));
        val[0] = log1pf(fmaxf(s0 / cnt - 100.f, 0.f)) * 0.125f;
        val[1] = log1pf(fmaxf(s1 / cnt - 100.f, 0.f)) * 0.125f;
    }
    const size_t pix = (size_t)ty * kT + tx;
    bf16 *o = x0 + pix * kC0;
    o[0] = __float2bfloat16(val[0]);
    o[1] = __float2bfloat16(val[1]);
    for (int c = 2; c < kC0; c++) o[c] = __float2bfloat16(0.f);
    if (thumbs) {
        thumbs[pix] = val[0];
        thumbs[kPix + pix] = val[1];
    }
}

// ------------------------------------------------------------ convolution
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// out[y][x][co] = epilogue(sum_{ky,kx,ci} in[y+ky-1][x+kx-1][ci] * W[ky][kx][ci][co])
// MODE 0: + bias, ReLU.  MODE 1: * (mask[y][x][co] > 0)  (input gradient).
template <int CIN, int MODE>
__global__ void __launch_bounds__(256) conv3x3_mma_kernel(const bf16 *__restrict__ in, const bf16 *__restrict__ wB,
                                                          const float *__restrict__ bias, const bf16 *__restrict__ mask,
                                                          bf16 *__restrict__ out) {
    constexpr int TW = 16, TH = 8, CP = CIN + 8;  // +8: conflict-free fragment loads
    __shared__ __align__(16) bf16 tile[TH + 2][TW + 2][CP];
    __shared__ __align__(16) bf16 wsm[9][kCh][CP];
    const int b = blockIdx.z, x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const bf16 *inb = in + (size_t)b * kPix * CIN;
    for (int i = threadIdx.x; i < (TH + 2) * (TW + 2) * (CIN / 2); i += blockDim.x) {
        const int c2 = i % (CIN / 2), pix = i / (CIN / 2);
        const int ty = pix / (TW + 2), tx = pix % (TW + 2);
        const int y = y0 + ty - 1, x = x0 + tx - 1;
        uint32_t v = 0;
        if (y >= 0 && y < kT && x >= 0 && x < kT) v = *reinterpret_cast<const uint32_t *>(inb + ((size_t)y * kT + x) * CIN + 2 * c2);
        *reinterpret_cast<uint32_t *>(&tile[ty][tx][2 * c2]) = v;
    }
    for (int i = threadIdx.x; i < 9 * kCh * (CIN / 2); i += blockDim.x) {
        const int c2 = i % (CIN / 2), r = i / (CIN / 2);
        *reinterpret_cast<uint32_t *>(&wsm[r / kCh][r % kCh][2 * c2]) = *reinterpret_cast<const uint32_t *>(wB + (size_t)r * CIN + 2 * c2);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[j][q] = 0.f;
#pragma unroll
    for (int kk = 0; kk < 9; kk++) {
        const int ky = kk / 3, kx = kk % 3;
#pragma unroll
        for (int cb = 0; cb < CIN; cb += 16) {
            uint32_t a[4];
            a[0] = *reinterpret_cast<const uint32_t *>(&tile[w + ky][g + kx][cb + 2 * t]);
            a[1] = *reinterpret_cast<const uint32_t *>(&tile[w + ky][g + 8 + kx][cb + 2 * t]);
            a[2] = *reinterpret_cast<const uint32_t *>(&tile[w + ky][g + kx][cb + 2 * t + 8]);
            a[3] = *reinterpret_cast<const uint32_t *>(&tile[w + ky][g + 8 + kx][cb + 2 * t + 8]);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&wsm[kk][j * 8 + g][cb + 2 * t]);
                const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&wsm[kk][j * 8 + g][cb + 2 * t + 8]);
                mma_bf16(acc[j], a, b0, b1);
            }
        }
    }
    const int y = y0 + w;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int co = j * 8 + 2 * t;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int x = x0 + g + 8 * h;
            const size_t pix = (size_t)b * kPix + (size_t)y * kT + x;
            float v0 = acc[j][2 * h], v1 = acc[j][2 * h + 1];
            if (MODE == 0) {
                v0 = fmaxf(v0 + bias[co], 0.f);
                v1 = fmaxf(v1 + bias[co + 1], 0.f);
            } else {
                const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + pix * kCh + co);
                if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
            }
            *reinterpret_cast<__nv_bfloat162 *>(out + pix * kCh + co) = __floats2bfloat162_rn(v0, v1);
        }
    }
}

// ---------------------------------------------------------------- head
__global__ void gap_partial_kernel(const bf16 *__restrict__ act, float *__restrict__ part) {
    __shared__ float sh[8][kCh];
    const int b = blockIdx.y, chunk = blockIdx.x;  // 64 chunks of 1024 positions
    const int c = threadIdx.x & 31, r = threadIdx.x >> 5;
    const bf16 *base = act + ((size_t)b * kPix + (size_t)chunk * 1024) * kCh;
    float s = 0.f;
    for (int p = r; p < 1024; p += 8) s += __bfloat162float(base[(size_t)p * kCh + c]);
    sh[r][c] = s;
    __syncthreads();
    if (r == 0) {
        float t = 0.f;
        for (int k = 0; k < 8; k++) t += sh[k][c];
        part[((size_t)b * 64 + chunk) * kCh + c] = t;
    }
}

// One warp per frame: pool, logits, softmax; with labels also the loss and
// d loss / d logits (batch mean).
__global__ void head_kernel(const float *__restrict__ part, const float *__restrict__ params, size_t off_wl, size_t off_bl,
                            int K, int nb, float *__restrict__ gap, float *__restrict__ probs, const int32_t *__restrict__ labels,
                            float *__restrict__ dz, float *__restrict__ loss) {
    const int b = blockIdx.x, lane = threadIdx.x;
    float gc = 0.f;
    for (int k = 0; k < 64; k++) gc += part[((size_t)b * 64 + k) * kCh + lane];
    gc *= 1.f / (float)kPix;
    gap[b * kCh + lane] = gc;
    float lg[2];
    lg[0] = lane < K ? params[off_bl + lane] : -INFINITY;
    lg[1] = lane + 32 < K ? params[off_bl + lane + 32] : -INFINITY;
    for (int c = 0; c < kCh; c++) {  // every lane runs every shuffle
        const float gv = __shfl_sync(LFC_FULL, gc, c);
        if (lane < K) lg[0] += gv * params[off_wl + (size_t)c * K + lane];
        if (lane + 32 < K) lg[1] += gv * params[off_wl + (size_t)c * K + lane + 32];
    }
    float mx = fmaxf(lg[0], lg[1]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(LFC_FULL, mx, o));
    float e[2], s = 0.f;
    for (int h = 0; h < 2; h++) {
        e[h] = (lane + 32 * h < K) ? __expf(lg[h] - mx) : 0.f;
        s += e[h];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(LFC_FULL, s, o);
    for (int h = 0; h < 2; h++) {
        const int k = lane + 32 * h;
        if (k < K) {
            const float p = e[h] / s;
            probs[(size_t)b * K + k] = p;
            if (labels) {
                const int lab = labels[b];
                dz[(size_t)b * K + k] = (p - (k == lab ? 1.f : 0.f)) / (float)nb;
                if (k == lab) loss[b] = -logf(fmaxf(p, 1e-30f));
            }
        }
    }
}

// d wl, d bl (sums over the batch of dz, already divided by the batch) and
// d gap = wl dz per frame.
__global__ void head_backward_kernel(const float *__restrict__ gap, const float *__restrict__ dz, const float *__restrict__ params,
                                     float *__restrict__ grads, size_t off_wl, size_t off_bl, int K, int nb, float *__restrict__ dg) {
    for (int i = threadIdx.x; i < kCh * K; i += blockDim.x) {
        const int c = i / K, k = i % K;
        float s = 0.f;
        for (int b = 0; b < nb; b++) s += gap[b * kCh + c] * dz[(size_t)b * K + k];
        grads[off_wl + i] = s;
    }
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nb; b++) s += dz[(size_t)b * K + k];
        grads[off_bl + k] = s;
    }
    for (int i = threadIdx.x; i < nb * kCh; i += blockDim.x) {
        const int b = i / kCh, c = i % kCh;
        float s = 0.f;
        for (int k = 0; k < K; k++) s += params[off_wl + (size_t)c * K + k] * dz[(size_t)b * K + k];
        dg[i] = s;
    }
}

// gradient at the last convolution's pre-activation: pool gradient through ReLU
__global__ void dpre_last_kernel(const float *__restrict__ dg, const bf16 *__restrict__ act, bf16 *__restrict__ dpre, int nb) {
    const size_t total = (size_t)nb * kPix * kCh;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % kCh);
        const size_t b = i / ((size_t)kPix * kCh);
        const float v = __bfloat162float(act[i]) > 0.f ? dg[b * kCh + c] * (1.f / (float)kPix) : 0.f;
        dpre[i] = __float2bfloat16(v);
    }
}

// dW[ky][kx][ci][co] += sum over a band of rows of in[y+ky-1][x+kx-1][ci] * dpre[y][x][co];
// db[co] += sum dpre. Tasks: (tap, 4 input channels, 4 output channels).
template <int CIN>
__global__ void __launch_bounds__(256) conv_wgrad_kernel(const bf16 *__restrict__ in, const bf16 *__restrict__ dpre,
                                                         float *__restrict__ dW, float *__restrict__ db, int rows, int cin_real) {
    constexpr int XH = kT / 2;  // half a row per step keeps shared memory under 48 KB
    __shared__ __align__(16) bf16 ins[3][XH + 2][CIN];
    __shared__ __align__(16) bf16 dps[XH][kCh];
    constexpr int NTASK = 9 * (CIN / 4) * (kCh / 4);
    constexpr int TPT = (NTASK + 255) / 256;
    const int b = blockIdx.y, y0 = blockIdx.x * rows;
    float acc[TPT][16];
    float bacc = 0.f;
#pragma unroll
    for (int q = 0; q < TPT; q++)
#pragma unroll
        for (int e = 0; e < 16; e++) acc[q][e] = 0.f;
    for (int y = y0; y < y0 + rows; y++) {
        for (int xh = 0; xh < kT; xh += XH) {
            for (int i = threadIdx.x; i < 3 * (XH + 2) * (CIN / 2); i += blockDim.x) {
                const int c2 = i % (CIN / 2), r = i / (CIN / 2), row = r / (XH + 2), col = r % (XH + 2);
                const int yy = y + row - 1, xx = xh + col - 1;
                uint32_t v = 0;
                if (yy >= 0 && yy < kT && xx >= 0 && xx < kT)
                    v = *reinterpret_cast<const uint32_t *>(in + (((size_t)b * kT + yy) * kT + xx) * CIN + 2 * c2);
                *reinterpret_cast<uint32_t *>(&ins[row][col][2 * c2]) = v;
            }
            for (int i = threadIdx.x; i < XH * (kCh / 2); i += blockDim.x) {
                const int c2 = i % (kCh / 2), x = i / (kCh / 2);
                *reinterpret_cast<uint32_t *>(&dps[x][2 * c2]) =
                    *reinterpret_cast<const uint32_t *>(dpre + (((size_t)b * kT + y) * kT + xh + x) * kCh + 2 * c2);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < TPT; q++) {
                const int task = threadIdx.x + q * 256;
                if (task >= NTASK) break;
                const int kk = task / ((CIN / 4) * (kCh / 4)), rem = task % ((CIN / 4) * (kCh / 4));
                const int ci4 = rem / (kCh / 4), co4 = rem % (kCh / 4);
                const int ky = kk / 3, kx = kk % 3;
                if (ci4 * 4 >= cin_real) continue;
                for (int x = 0; x < XH; x++) {
                    float a[4], d[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        a[e] = __bfloat162float(ins[ky][x + kx][ci4 * 4 + e]);
                        d[e] = __bfloat162float(dps[x][co4 * 4 + e]);
                    }
#pragma unroll
                    for (int i2 = 0; i2 < 4; i2++)
#pragma unroll
                        for (int j2 = 0; j2 < 4; j2++) acc[q][i2 * 4 + j2] = fmaf(a[i2], d[j2], acc[q][i2 * 4 + j2]);
                }
            }
            if (threadIdx.x < kCh)
                for (int x = 0; x < XH; x++) bacc += __bfloat162float(dps[x][threadIdx.x]);
            __syncthreads();
        }
    }
#pragma unroll
    for (int q = 0; q < TPT; q++) {
        const int task = threadIdx.x + q * 256;
        if (task >= NTASK) break;
        const int kk = task / ((CIN / 4) * (kCh / 4)), rem = task % ((CIN / 4) * (kCh / 4));
        const int ci4 = rem / (kCh / 4), co4 = rem % (kCh / 4);
        for (int i2 = 0; i2 < 4; i2++) {
            const int ci = ci4 * 4 + i2;
            if (ci >= cin_real) continue;
            for (int j2 = 0; j2 < 4; j2++)
                atomicAdd(&dW[((size_t)kk * cin_real + ci) * kCh + co4 * 4 + j2], acc[q][i2 * 4 + j2]);
        }
    }
    if (threadIdx.x < kCh) atomicAdd(&db[threadIdx.x], bacc);
}

// Master FP32 weights -> BF16 operands: forward [tap][co][ci_pad],
// input gradient [tap][ci][co] with the tap flipped (8 - tap).
__global__ void pack_weights_kernel(const float *__restrict__ params, size_t off_w, int cin, int cin_pad, bf16 *__restrict__ wf,
                                    bf16 *__restrict__ wd) {
    const int n = 9 * kCh * cin_pad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int kk = i / (kCh * cin_pad), r = i % (kCh * cin_pad), co = r / cin_pad, ci = r % cin_pad;
        const float v = ci < cin ? params[off_w + ((size_t)kk * cin + ci) * kCh + co] : 0.f;
        wf[i] = __float2bfloat16(v);
    }
    if (wd) {
        const int m = 9 * kCh * kCh;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
            const int kk = i / (kCh * kCh), r = i % (kCh * kCh), ci = r / kCh, co = r % kCh;
            wd[i] = __float2bfloat16(params[off_w + ((size_t)(8 - kk) * cin + ci) * kCh + co]);
        }
    }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                            size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// He-normal weights from a counter-based generator (splitmix64 + Box-Muller),
// zero biases.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void init_params_kernel(float *__restrict__ p, POff o, int K, uint64_t seed) {
    const size_t n = o.total;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float scale = 0.f;
        const int cin[4] = {2, kCh, kCh, kCh};
        for (int l = 0; l < 4; l++)
            if (i >= o.w[l] && i < o.b[l]) scale = sqrtf(2.f / (9.f * cin[l]));
        if (i >= o.wl && i < o.bl) scale = sqrtf(1.f / kCh);
        if (scale == 0.f) { p[i] = 0.f; continue; }
        const uint64_t r = splitmix64(seed * 0x100000001B3ull + i);
        const float u1 = ((float)(r >> 40) + 0.5f) * (1.f / 16777216.f);
        const float u2 = ((float)((r >> 16) & 0xFFFFFF) + 0.5f) * (1.f / 16777216.f);
        p[i] = scale * sqrtf(-2.f * logf(u1)) * cosf(6.28318530718f * u2);
    }
}

// Top-k candidate mask from the softmax; all candidates when the top
// probability is below tau. With k = 1 and a confident proposal the choice
// is written directly.
__global__ void propose_mask_kernel(const float *__restrict__ probs, int K, const uint8_t *__restrict__ class_ids, int topk,
                                    float tau, uint64_t *__restrict__ masks, int nb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const float *pb = probs + (size_t)b * K;
    uint64_t mk[4] = {0, 0, 0, 0};
    float top = 0.f;
    for (int k = 0; k < K; k++) top = fmaxf(top, pb[k]);
    if (top < tau) {
        for (int k = 0; k < K; k++) mk[class_ids[k] >> 6] |= 1ull << (class_ids[k] & 63);
    } else {
        uint64_t taken = 0;
        for (int r = 0; r < topk && r < K; r++) {
            int best = -1;
            for (int k = 0; k < K; k++)
                if (!((taken >> k) & 1) && (best < 0 || pb[k] > pb[best])) best = k;
            taken |= 1ull << best;
            mk[class_ids[best] >> 6] |= 1ull << (class_ids[best] & 63);
        }
    }
    for (int q = 0; q < 4; q++) masks[(size_t)b * 4 + q] = mk[q];
}

cudaError_t launch_propose_mask(const float *probs, int K, const uint8_t *class_ids, int topk, float tau, uint64_t *masks,
                                int nb, cudaStream_t s) {
    propose_mask_kernel<<<(nb + 127) / 128, 128, 0, s>>>(probs, K, class_ids, topk, tau, masks, nb);
    return cudaGetLastError();
}

}  // namespace lfc

// ================================================================ C ABI
using namespace lfc;

static int cnn_fail(lfc_cnn C, int code, const char *what, cudaError_t e = cudaSuccess) {
    if (C) {
        C->err = what;
        if (e != cudaSuccess) { C->err += ": "; C->err += cudaGetErrorString(e); }
    }
    return code;
}
#define CKC(x)                                                              \
    do {                                                                    \
        cudaError_t _e = (x);                                               \
        if (_e != cudaSuccess) return cnn_fail(C, LFC_ERR_CUDA, #x, _e);    \
    } while (0)

static void cnn_free(lfc_cnn C) {
    void *ptrs[] = {C->params, C->grads, C->m, C->v, C->wf[0], C->wf[1], C->wf[2], C->wf[3], C->wd[0], C->wd[1],
                    C->wd[2], C->wd[3], C->x0, C->act[0], C->act[1], C->act[2], C->act[3], C->dpre[0], C->dpre[1],
                    C->gap_part, C->gap, C->probs, C->dz, C->dg, C->loss};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

static cudaError_t pack_all(lfc_cnn C) {
    const int cin[4] = {2, kCh, kCh, kCh}, cpad[4] = {kC0, kCh, kCh, kCh};
    for (int l = 0; l < 4; l++)
        pack_weights_kernel<<<36, 256, 0, C->stream>>>(C->params, C->off.w[l], cin[l], cpad[l], C->wf[l], l > 0 ? C->wd[l] : nullptr);
    return cudaGetLastError();
}

extern "C" int lfc_cnn_create(int n_classes, int max_batch, uint64_t seed, void *cuda_stream, lfc_cnn *out) {
    if (!out || n_classes < 2 || n_classes > 64 || max_batch < 1) return LFC_ERR_INVALID_ARG;
    *out = nullptr;
    lfc_cnn C = new (std::nothrow) lfc_cnn_s();
    if (!C) return LFC_ERR_NOMEM;
    C->K = n_classes;
    C->max_batch = max_batch;
    C->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    C->off = param_offsets(n_classes);
    const size_t np = C->off.total, B = (size_t)max_batch;
    cudaError_t e = cudaSuccess;
    auto al = [&](void **p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    al((void **)&C->params, np * 4);
    al((void **)&C->grads, np * 4);
    al((void **)&C->m, np * 4);
    al((void **)&C->v, np * 4);
    const int cpad[4] = {kC0, kCh, kCh, kCh};
    for (int l = 0; l < 4; l++) {
        al((void **)&C->wf[l], (size_t)9 * kCh * cpad[l] * 2);
        if (l > 0) al((void **)&C->wd[l], (size_t)9 * kCh * kCh * 2);
    }
    al((void **)&C->x0, B * kPix * kC0 * 2);
    for (int l = 0; l < 4; l++) al((void **)&C->act[l], B * kPix * kCh * 2);
    for (int l = 0; l < 2; l++) al((void **)&C->dpre[l], B * kPix * kCh * 2);
    al((void **)&C->gap_part, B * 64 * kCh * 4);
    al((void **)&C->gap, B * kCh * 4);
    al((void **)&C->probs, B * n_classes * 4);
    al((void **)&C->dz, B * n_classes * 4);
    al((void **)&C->dg, B * kCh * 4);
    al((void **)&C->loss, B * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(C->m, 0, np * 4, C->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(C->v, 0, np * 4, C->stream);
    if (e == cudaSuccess) {
        init_params_kernel<<<64, 256, 0, C->stream>>>(C->params, C->off, n_classes, seed);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = pack_all(C);
    if (e == cudaSuccess) e = cudaStreamSynchronize(C->stream);
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        cnn_free(C);
        delete C;
        return oom ? LFC_ERR_NOMEM : LFC_ERR_CUDA;
    }
    *out = C;
    return LFC_OK;
}

extern "C" void lfc_cnn_destroy(lfc_cnn C) {
    if (!C) return;
    cudaStreamSynchronize(C->stream);
    cnn_free(C);
    delete C;
}

extern "C" const char *lfc_cnn_last_error(lfc_cnn C) { return C ? C->err.c_str() : "null network"; }

extern "C" size_t lfc_cnn_param_count(lfc_cnn C) { return C ? C->off.total : 0; }

extern "C" int lfc_cnn_set_params(lfc_cnn C, const float *h_params, size_t n) {
    if (!C || !h_params || n != C->off.total) return cnn_fail(C, LFC_ERR_INVALID_ARG, "lfc_cnn_set_params: size");
    CKC(cudaMemcpy(C->params, h_params, n * 4, cudaMemcpyHostToDevice));
    CKC(pack_all(C));
    CKC(cudaStreamSynchronize(C->stream));
    return LFC_OK;
}

extern "C" int lfc_cnn_get_params(lfc_cnn C, float *h_params, float *h_grads, size_t n) {
    if (!C || n != C->off.total) return cnn_fail(C, LFC_ERR_INVALID_ARG, "lfc_cnn_get_params: size");
    CKC(cudaStreamSynchronize(C->stream));
    if (h_params) CKC(cudaMemcpy(h_params, C->params, n * 4, cudaMemcpyDeviceToHost));
    if (h_grads) CKC(cudaMemcpy(h_grads, C->grads, n * 4, cudaMemcpyDeviceToHost));
    return LFC_OK;
}

static int cnn_thumbs(lfc_cnn C, const lfc_frame *frames, int n, float *d_thumbs) {
    for (int i = 0; i < n; i++) {
        const lfc_frame &f = frames[i];
        if (!f.data || f.pitch <= 0 || f.width % f.pitch || f.height % f.pitch) return cnn_fail(C, LFC_ERR_INVALID_ARG, "frame");
        FrameDev F;
        F.X = f.data;
        F.prev = nullptr;
        F.W = f.width;
        F.H = f.height;
        F.p = f.pitch;
        F.Nx = f.width / f.pitch;
        F.Ny = f.height / f.pitch;
        const int bs = (std::max(F.W, F.H) + kT - 1) / kT;
        thumb_kernel<<<dim3(1, kT), kT, 0, C->stream>>>(F, bs, C->x0 + (size_t)i * kPix * kC0,
                                                        d_thumbs ? d_thumbs + (size_t)i * 2 * kPix : nullptr);
    }
    CKC(cudaGetLastError());
    return LFC_OK;
}

extern "C" int lfc_cnn_thumbnails(lfc_cnn C, const lfc_frame *h_frames, int n, float *d_thumbs) {
    if (!C || !h_frames || n < 1 || n > C->max_batch) return cnn_fail(C, LFC_ERR_INVALID_ARG, "lfc_cnn_thumbnails: n");
    return cnn_thumbs(C, h_frames, n, d_thumbs);
}

// Caller FP32 thumbnails (planar n x 2 x 256 x 256) into the network input
// (NHWC BF16, channels 2..15 zero), round to nearest even.
__global__ void set_thumbs_kernel(const float *__restrict__ th, int n, bf16 *__restrict__ x0) {
    const size_t total = (size_t)n * kPix;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / kPix, pix = i % kPix;
        bf16 *o = x0 + i * kC0;
        o[0] = __float2bfloat16(th[(b * 2) * kPix + pix]);
        o[1] = __float2bfloat16(th[(b * 2 + 1) * kPix + pix]);
        for (int c = 2; c < kC0; c++) o[c] = __float2bfloat16(0.f);
    }
}

extern "C" int lfc_cnn_set_thumbnails(lfc_cnn C, const float *d_thumbs, int n) {
    if (!C || !d_thumbs || n < 1 || n > C->max_batch) return cnn_fail(C, LFC_ERR_INVALID_ARG, "lfc_cnn_set_thumbnails");
    set_thumbs_kernel<<<(unsigned)std::min<size_t>(4096, ((size_t)n * kPix + 255) / 256), 256, 0, C->stream>>>(d_thumbs, n, C->x0);
    CKC(cudaGetLastError());
    return LFC_OK;
}

static int cnn_forward(lfc_cnn C, int n) {
    cudaStream_t s = C->stream;
    dim3 grid(kT / 16, kT / 8, n);
    conv3x3_mma_kernel<kC0, 0><<<grid, 256, 0, s>>>(C->x0, C->wf[0], C->params + C->off.b[0], nullptr, C->act[0]);
    for (int l = 1; l < 4; l++)
        conv3x3_mma_kernel<kCh, 0><<<grid, 256, 0, s>>>(C->act[l - 1], C->wf[l], C->params + C->off.b[l], nullptr, C->act[l]);
    gap_partial_kernel<<<dim3(64, n), 256, 0, s>>>(C->act[3], C->gap_part);
    CKC(cudaGetLastError());
    return LFC_OK;
}

extern "C" int lfc_cnn_forward(lfc_cnn C, int n, float *d_probs) {
    if (!C || n < 1 || n > C->max_batch) return cnn_fail(C, LFC_ERR_INVALID_ARG, "lfc_cnn_forward: n");
    int r = cnn_forward(C, n);
    if (r) return r;
    head_kernel<<<n, 32, 0, C->stream>>>(C->gap_part, C->params, C->off.wl, C->off.bl, C->K, n, C->gap,
                                        d_probs ? d_probs : C->probs, nullptr, nullptr, nullptr);
    CKC(cudaGetLastError());
    return LFC_OK;
}

extern "C" int lfc_cnn_backward(lfc_cnn C, int n, const int32_t *d_labels, float *d_loss) {
    if (!C || !d_labels || n < 1 || n > C->max_batch) return cnn_fail(C, LFC_ERR_INVALID_ARG, "lfc_cnn_backward");
    cudaStream_t s = C->stream;
    int r = cnn_forward(C, n);
    if (r) return r;
    head_kernel<<<n, 32, 0, s>>>(C->gap_part, C->params, C->off.wl, C->off.bl, C->K, n, C->gap, C->probs, d_labels, C->dz,
                                 d_loss ? d_loss : C->loss);
    CKC(cudaMemsetAsync(C->grads, 0, C->off.total * 4, s));
    head_backward_kernel<<<1, 256, 0, s>>>(C->gap, C->dz, C->params, C->grads, C->off.wl, C->off.bl, C->K, n, C->dg);
    dpre_last_kernel<<<1216, 256, 0, s>>>(C->dg, C->act[3], C->dpre[1], n);
    constexpr int rows = 16;
    dim3 wgrid(kT / rows, n);
    dim3 grid(kT / 16, kT / 8, n);
    int cur = 1;
    for (int l = 3; l >= 0; l--) {
        if (l > 0)
            conv_wgrad_kernel<kCh><<<wgrid, 256, 0, s>>>(C->act[l - 1], C->dpre[cur], C->grads + C->off.w[l],
                                                           C->grads + C->off.b[l], rows, kCh);
        else
            conv_wgrad_kernel<kC0><<<wgrid, 256, 0, s>>>(C->x0, C->dpre[cur], C->grads + C->off.w[0], C->grads + C->off.b[0],
                                                           rows, 2);
        if (l > 0) {
            conv3x3_mma_kernel<kCh, 1><<<grid, 256, 0, s>>>(C->dpre[cur], C->wd[l], nullptr, C->act[l - 1], C->dpre[cur ^ 1]);
            cur ^= 1;
        }
    }
    CKC(cudaGetLastError());
    return LFC_OK;
}

extern "C" int lfc_cnn_adam_step(lfc_cnn C, float lr, float beta1, float beta2, float eps) {
    if (!C) return LFC_ERR_INVALID_ARG;
    C->step++;
    const float c1 = 1.f - powf(beta1, (float)C->step), c2 = 1.f - powf(beta2, (float)C->step);
    adam_kernel<<<64, 256, 0, C->stream>>>(C->params, C->grads, C->m, C->v, C->off.total, lr, beta1, beta2, eps, c1, c2);
    CKC(cudaGetLastError());
    CKC(pack_all(C));
    return LFC_OK;
}

// used by the plan's proposal path
namespace lfc {
int cnn_propose(lfc_cnn C, const lfc_frame *frames, int n, const uint8_t *d_class_ids, int topk, float tau, uint64_t *d_masks,
                cudaStream_t s) {
    cudaStream_t home = C->stream;
    C->stream = s;
    int r = LFC_OK;
    for (int f0 = 0; f0 < n && r == LFC_OK; f0 += C->max_batch) {
        const int nb = std::min(C->max_batch, n - f0);
        r = cnn_thumbs(C, frames + f0, nb, nullptr);
        if (r == LFC_OK) r = lfc_cnn_forward(C, nb, nullptr);
        if (r == LFC_OK) {
            const cudaError_t e = launch_propose_mask(C->probs, C->K, d_class_ids, topk, tau, d_masks + (size_t)f0 * 4, nb, s);
            if (e != cudaSuccess) r = cnn_fail(C, LFC_ERR_CUDA, "propose", e);
        }
    }
    C->stream = home;
    return r;
}
int cnn_classes(lfc_cnn C) { return C ? C->K : 0; }
int cnn_max_batch(lfc_cnn C) { return C ? C->max_batch : 0; }
}  // namespace lfc

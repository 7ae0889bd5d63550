// Learned right preconditioner: linear 3-level U-Net (see unet.h).
//
// A 3-D grid is handled as the image of its nz * ny rows (z, y) by nx columns,
// cut into slices of ny rows: the 3x3 convolutions read only rows of their
// own slice, and pooling / upsampling pair slices as well as rows and columns.
//
// Convolutions: implicit GEMM per 16x8 pixel tile, M = 128 pixels (8 warps x 16),
// N = output channels, K = 9 taps x input channels, using
// mma.sync.m16n8k16.row.col.f32.bf16.bf16.f32 with ldmatrix fragments from
// shared memory (input tile with a one-pixel halo, NHWC, and the layer's
// weights [tap][cout][cin], resident for the CTA's lifetime).  The backward pass w.r.t. the input is the same
// kernel with flipped, transposed weights; the weight gradient is a float32
// reduction over pixel tiles (CUDA cores) with one atomic add per weight and
// tile.
#include <atomic>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "unet.h"

namespace jfnk {
namespace {

constexpr int NL = 9;     // layers
enum { L0a, L0b, L1a, L1b, L2a, L2b, L1c, L0c, L0d };
constexpr int CIN[NL] = {16, 16, 16, 32, 32, 64, 96, 48, 16};
constexpr int COUT[NL] = {16, 16, 32, 32, 64, 64, 32, 16, 16};
constexpr int KSZ[NL] = {3, 3, 3, 3, 3, 3, 3, 3, 1};

typedef __nv_bfloat16 bf16;

constexpr int MAXF = 5;   // field planes of a 3-D state (u, v, w, theta, p); 2-D has 4

// Field balance of the network: it sees B x and returns B N(x).
struct Bal {
    float b[MAXF], inv[MAXF];
    int nf;
};

// Geometry of one level of the network.  A 2-D grid is one slice of H rows
// (z) by Wd columns (x).  A 3-D grid [z][y][x] is a stack of H / Hs slices of
// Hs rows (y) each: row r holds (z, y) = (r / Hs, r % Hs).  The 3x3
// convolutions act within a slice (zero padding at its first and last rows);
// pooling and upsampling pair slices 2z, 2z+1 as well when d3 = 1.
struct Lv {
    int H, Wd, Hs, d3;
};

// row of the coarser level holding the parent of fine row r
__host__ __device__ __forceinline__ int coarse_row(int r, const Lv& f) {
    const int z = r / f.Hs, y = r - z * f.Hs;
    return (z >> 1) * (f.Hs >> 1) + (y >> 1);
}

// fine row of child (dz, dy) of coarse row q (f: the fine level)
__host__ __device__ __forceinline__ int fine_row(int q, int dz, int dy, const Lv& f) {
    const int hc = f.Hs >> 1;
    const int z = q / hc, y = q - z * hc;
    return (2 * z + dz) * f.Hs + 2 * y + dy;
}

// convolution tile: CONV_TH rows x CONV_TW columns, one warp per pair of rows
constexpr int CONV_TW = 8, CONV_TH = 16, CONV_THREADS = 32 * CONV_TH / 2;

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------- convolution
// out[p][co] = sum_tap sum_ci W[tap][co][ci] in[p + off(tap)][ci] (zero padding).
// in / out are NHWC with pixel strides istr / ostr (channels) and channel offsets.
//
// Persistent CTAs: the layer's weights are copied to shared memory once per
// CTA, which then walks over CONV_TH x CONV_TW pixel tiles with a stride of
// gridDim.x, prefetching the next tile's input (with its halo) by cp.async
// while the tensor cores work on the current one.  Shared rows are padded by
// 8 channels so that the ldmatrix row addresses of a fragment fall in
// distinct bank groups.  Warp w owns pixel rows 2w and 2w+1 of the tile: the
// 16 rows of its mma A fragment are (2w, 0..7) and (2w+1, 0..7).
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// Programmatic dependent launch between the layers: a convolution is launched
// before its predecessor has finished, prefetches its weights (which do not
// depend on the predecessor), and waits (griddepcontrol.wait) before it reads
// the previous layer's output or the skip flag; each CTA releases the next
// layer's launch (griddepcontrol.launch_dependents) when it starts its last tile.
__device__ __forceinline__ void net_pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void net_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t net_launch(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// 16-byte global -> shared copy; src_bytes = 0 writes zeros (src is not read).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <int CI, int CO, int KS>
struct ConvShape {
    static constexpr int HP = KS / 2;
    static constexpr int IH = CONV_TH + 2 * HP, IW = CONV_TW + 2 * HP;
    static constexpr int CIP = CI + 8;                       // padded channel stride (elements)
    static constexpr int W_ELEMS = KS * KS * CO * CIP;
    static constexpr int X_ELEMS = IH * IW * CIP;
    static constexpr size_t SMEM = sizeof(bf16) * (size_t)(W_ELEMS + 2 * X_ELEMS);
};

// Input staging modes of a convolution (what the CTA copies into its tile):
//   IN_NHWC   a bfloat16 NHWC tensor (pixel stride astr, channel offset aoff)
//   IN_PACK   B x from four float32 field planes (channels 4.. are zero)
//   IN_POOL   2x2 average of a tensor of twice the grid's size
//   IN_UPCAT  [nearest upsampling of a half-size tensor a (CU channels) | b]
// Output modes: OUT_BF16 / OUT_F32 NHWC (pixel stride ostr, channel offset
// ooff), OUT_PLANES: channels 0..3 times B^-1 into four float32 planes,
// stored or added.
enum { IN_NHWC = 0, IN_PACK = 1, IN_POOL = 2, IN_UPCAT = 3 };
enum { OUT_BF16 = 0, OUT_F32 = 1, OUT_PLANES = 2 };

struct ConvIn {
    const bf16* a;
    int astr, aoff;
    const bf16* b;      // IN_UPCAT: the full-size part
    int bstr, boff;
    const float* x;     // IN_PACK: field planes
};

struct ConvOut {
    void* o;
    int ostr, ooff;
    int accumulate;     // OUT_PLANES
};

// LAYOUT 0: pixel-major rows padded to CIP channels (ldmatrix operands of conv_mma).
// LAYOUT 1: the canonical K-major, no-swizzle operand layout of tcgen05.mma
// (conv_tc): for every tile row iy and 8-channel group v, the IW pixels' 16-byte
// groups lie contiguously, at iy * (CI/8) * IW * 16 + v * IW * 16 + ix * 16 bytes.
template <int CI, int IH, int IW, int CIP, int INMODE, int CU, int LAYOUT = 0>
__device__ __forceinline__ void stage_tile(const ConvIn& in, const Bal& bal, const Lv& g, int y0, int x0, int hp,
                                           uint32_t xs_addr) {
    constexpr int VPP = CI / 8;
    const int H = g.H, Wd = g.Wd;
    const int sy0 = (y0 / g.Hs) * g.Hs;              // first row of the tile's slice
    const int sy1 = min(sy0 + g.Hs, H);
    for (int idx = threadIdx.x; idx < IH * IW * VPP; idx += blockDim.x) {
        const int pix = idx / VPP, v = idx - pix * VPP;
        const int iy = pix / IW, ix = pix - iy * IW;
        const int gy = y0 + iy - hp, gx = x0 + ix - hp;
        const bool ok = gy >= sy0 && gy < sy1 && gx >= 0 && gx < Wd;
        const uint32_t dst = LAYOUT == 0 ? xs_addr + (uint32_t)((pix * CIP + v * 8) * sizeof(bf16))
                                         : xs_addr + (uint32_t)(((iy * VPP + v) * IW + ix) * 16);
        if constexpr (INMODE == IN_NHWC) {
            const bf16* src = ok ? in.a + ((size_t)gy * Wd + gx) * in.astr + in.aoff + v * 8 : in.a;
            cp_async16(dst, src, ok ? 16 : 0);
        } else if constexpr (INMODE == IN_UPCAT) {
            const bf16* src;
            if (v * 8 < CU)
                src = ok ? in.a + ((size_t)coarse_row(gy, g) * (Wd >> 1) + (gx >> 1)) * in.astr + in.aoff + v * 8
                         : in.a;
            else
                src = ok ? in.b + ((size_t)gy * Wd + gx) * in.bstr + in.boff + (v * 8 - CU) : in.b;
            cp_async16(dst, src, ok ? 16 : 0);
        } else {
            __align__(16) bf16 val[8];
            if constexpr (INMODE == IN_PACK) {
                const size_t npix = (size_t)H * Wd;
#pragma unroll
                for (int c = 0; c < 8; ++c) val[c] = __float2bfloat16(0.f);
                if (v == 0 && ok) {
#pragma unroll
                    for (int c = 0; c < MAXF; ++c)
                        if (c < bal.nf)
                            val[c] = __float2bfloat16(bal.b[c] * in.x[(size_t)c * npix + (size_t)gy * Wd + gx]);
                }
            } else {   // IN_POOL: same arithmetic as the avgpool2 kernel (children summed in (dz, d) order)
                const Lv f{2 * g.H * (1 + g.d3), 2 * Wd, 2 * g.Hs, g.d3};     // the fine level
                const int W2 = 2 * Wd;
                float sum[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) sum[c] = 0.f;
                if (ok) {
                    for (int dz = 0; dz <= g.d3; ++dz)
#pragma unroll
                        for (int d = 0; d < 4; ++d) {
                            const uint4 q = *reinterpret_cast<const uint4*>(
                                in.a + ((size_t)fine_row(gy, dz, d / 2, f) * W2 + 2 * gx + d % 2) * in.astr + in.aoff +
                                v * 8);
                            const bf16* e = reinterpret_cast<const bf16*>(&q);
#pragma unroll
                            for (int c = 0; c < 8; ++c) sum[c] += __bfloat162float(e[c]);
                        }
                }
                const float wgt = g.d3 ? 0.125f : 0.25f;
#pragma unroll
                for (int c = 0; c < 8; ++c) val[c] = __float2bfloat16(wgt * sum[c]);
            }
            asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};\n" ::"r"(dst),
                         "r"(reinterpret_cast<uint32_t*>(val)[0]), "r"(reinterpret_cast<uint32_t*>(val)[1]),
                         "r"(reinterpret_cast<uint32_t*>(val)[2]), "r"(reinterpret_cast<uint32_t*>(val)[3]));
        }
    }
}

template <int CI, int CO, int KS, int INMODE, int OUTMODE, int CU>
__global__ void __launch_bounds__(CONV_THREADS)
conv_mma(ConvIn in, Bal bal, const bf16* __restrict__ W, ConvOut out, Lv lv, const int* skip) {
    using S = ConvShape<CI, CO, KS>;
    constexpr int HP = S::HP, IW = S::IW, IH = S::IH, CIP = S::CIP;
    extern __shared__ __align__(16) unsigned char sm[];
    bf16* ws = reinterpret_cast<bf16*>(sm);
    const uint32_t ws_addr = (uint32_t)__cvta_generic_to_shared(ws);
    const uint32_t xs_addr0 = ws_addr + (uint32_t)(S::W_ELEMS * sizeof(bf16));
    const uint32_t xs_bytes = (uint32_t)(S::X_ELEMS * sizeof(bf16));
    const int H = lv.H, Wd = lv.Wd;
    const int ntx = (Wd + CONV_TW - 1) / CONV_TW, nty = (H + CONV_TH - 1) / CONV_TH;
    const int ntiles = ntx * nty;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    // weights (group 0, before the wait for the previous layer) and the first tile (group 1)
    for (int idx = threadIdx.x; idx < KS * KS * CO * (CI / 8); idx += blockDim.x) {
        const int row = idx / (CI / 8), v = idx - row * (CI / 8);
        cp_async16(ws_addr + (uint32_t)((row * CIP + v * 8) * sizeof(bf16)), W + (size_t)row * CI + v * 8, 16);
    }
    cp_async_commit();
    net_pdl_wait();
    if (skip != nullptr && *skip) {
        cp_async_wait<0>();
        return;
    }
    stage_tile<CI, IH, IW, CIP, INMODE, CU>(in, bal, lv, (tile / ntx) * CONV_TH, (tile % ntx) * CONV_TW, HP,
                                            xs_addr0);
    cp_async_commit();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    // ldmatrix row of this lane: A rows 0-7 = (2w, 0..7), rows 8-15 = (2w+1, 0..7); k half = lane >> 4
    const int arow = lane & 15;
    const int apy = 2 * warp + (arow >> 3), apx = arow & 7;
    const int akoff = (lane >> 4) * 8;
    int buf = 0;
    for (; tile < ntiles; tile += gridDim.x, buf ^= 1) {
        const int next = tile + gridDim.x;
        if (next >= ntiles) net_pdl_trigger();     // last tile of this CTA
        if (next < ntiles)
            stage_tile<CI, IH, IW, CIP, INMODE, CU>(in, bal, lv, (next / ntx) * CONV_TH, (next % ntx) * CONV_TW,
                                                    HP, xs_addr0 + (buf ^ 1) * xs_bytes);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const uint32_t xs_addr = xs_addr0 + buf * xs_bytes;
        float acc[CO / 8][4];
#pragma unroll
        for (int nb = 0; nb < CO / 8; ++nb)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[nb][q] = 0.f;
#pragma unroll
        for (int tap = 0; tap < KS * KS; ++tap) {
            const int dy = tap / KS - HP, dx = tap % KS - HP;
            const uint32_t a_base =
                xs_addr + (uint32_t)((((apy + HP + dy) * IW + (apx + HP + dx)) * CIP + akoff) * sizeof(bf16));
#pragma unroll
            for (int c = 0; c < CI / 16; ++c) {
                uint32_t a0, a1, a2, a3;
                ldsm_x4(a_base + c * 32, a0, a1, a2, a3);
#pragma unroll
                for (int nb = 0; nb < CO / 8; nb += 2) {   // CO / 8 is even for every layer
                    // matrices: (nb, k0), (nb, k8), (nb+1, k0), (nb+1, k8)
                    uint32_t b0, b1, b2, b3;
                    const int i = lane >> 3;
                    const int co = (nb + (i >> 1)) * 8 + (lane & 7);
                    ldsm_x4(ws_addr + (uint32_t)(((tap * CO + co) * CIP + c * 16 + (i & 1) * 8) * sizeof(bf16)), b0,
                            b1, b2, b3);
                    mma16816(acc[nb], a0, a1, a2, a3, b0, b1);
                    mma16816(acc[nb + 1], a0, a1, a2, a3, b2, b3);
                }
            }
        }
        const int y0 = (tile / ntx) * CONV_TH, x0 = (tile % ntx) * CONV_TW;
        const int gyA = y0 + 2 * warp, gyB = gyA + 1, gx = x0 + g;
        if (gx < Wd) {
            if constexpr (OUTMODE == OUT_PLANES) {
                // channels 2t, 2t+1 of block 0: lanes t = 0, 1, 2 hold the field channels
                if (t < 3) {
                    float* o = reinterpret_cast<float*>(out.o);
                    const size_t npix = (size_t)H * Wd;
                    const float inv[2] = {bal.inv[min(2 * t, MAXF - 1)], bal.inv[min(2 * t + 1, MAXF - 1)]};
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const int ch = 2 * t + q;
                        if (ch >= bal.nf) continue;
                        if (gyA < H) {
                            float* d = o + (size_t)ch * npix + (size_t)gyA * Wd + gx;
                            const float v = acc[0][q] * inv[q];
                            *d = out.accumulate ? *d + v : v;
                        }
                        if (gyB < H) {
                            float* d = o + (size_t)ch * npix + (size_t)gyB * Wd + gx;
                            const float v = acc[0][2 + q] * inv[q];
                            *d = out.accumulate ? *d + v : v;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int nb = 0; nb < CO / 8; ++nb) {
                    const int co = nb * 8 + 2 * t;
                    if constexpr (OUTMODE == OUT_F32) {
                        float* o = reinterpret_cast<float*>(out.o);
                        if (gyA < H)
                            *reinterpret_cast<float2*>(o + ((size_t)gyA * Wd + gx) * out.ostr + out.ooff + co) =
                                make_float2(acc[nb][0], acc[nb][1]);
                        if (gyB < H)
                            *reinterpret_cast<float2*>(o + ((size_t)gyB * Wd + gx) * out.ostr + out.ooff + co) =
                                make_float2(acc[nb][2], acc[nb][3]);
                    } else {
                        bf16* o = reinterpret_cast<bf16*>(out.o);
                        if (gyA < H)
                            *reinterpret_cast<__nv_bfloat162*>(o + ((size_t)gyA * Wd + gx) * out.ostr + out.ooff + co) =
                                __floats2bfloat162_rn(acc[nb][0], acc[nb][1]);
                        if (gyB < H)
                            *reinterpret_cast<__nv_bfloat162*>(o + ((size_t)gyB * Wd + gx) * out.ostr + out.ooff + co) =
                                __floats2bfloat162_rn(acc[nb][2], acc[nb][3]);
                    }
                }
            }
        }
        __syncthreads();   // the next prefetch overwrites this buffer
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------- tcgen05 convolution
// The same convolution as conv_mma on the fifth-generation tensor cores: one
// CTA computes a CONV_TH x CONV_TW = 16 x 8 pixel tile as the M = 128 rows of
// the implicit GEMM D[pixel][co] = sum_tap sum_ci A_tap[pixel][ci] W[tap][co][ci].
// The staged input tile (halo included) is kept in the canonical K-major,
// no-swizzle layout (stage_tile LAYOUT 1), so the A operand of tap (ky, kx) is
// the same tile at a descriptor offset of ky rows and kx pixels: no im2col
// copy.  The layer's weights stay resident as the B operand (K-major core
// matrices).  One thread issues the K / 16 tcgen05.mma.kind::f16 instructions
// (bfloat16 operands, float32 accumulation) of a tile into one of two TMEM
// accumulators and commits them to an mbarrier; while they run, the CTA
// stages the next tile into the other input buffer; then every warp reads its
// 32 TMEM lanes (= 32 pixels) with tcgen05.ld and writes the output.  Waits on
// the mbarrier are bounded: on a time-out the CTA records an error, lets its
// copies drain, frees its TMEM and returns.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of tcgen05.mma: start address, leading
// (K-direction core matrix) and stride (M/N-direction core matrix) byte
// offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D float32, A and B bfloat16, both K-major, M x N.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ bool mbar_test(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(addr), "r"(parity)
                 : "memory");
    return ok != 0;
}

// 8 float32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <int CI, int CO, int KS>
struct TcShape {
    static constexpr int HP = KS / 2;
    static constexpr int IH = CONV_TH + 2 * HP, IW = CONV_TW + 2 * HP;
    static constexpr int C8 = CI / 8;
    static constexpr uint32_t A_LBO = IW * 16;              // next 8 input channels
    static constexpr uint32_t A_SBO = C8 * IW * 16;         // next pixel row of the tile
    static constexpr uint32_t A_BYTES = IH * A_SBO;
    static constexpr uint32_t B_LBO = 128;                  // next 8 input channels
    static constexpr uint32_t B_SBO = C8 * 128;             // next 8 output channels
    static constexpr uint32_t B_TAP = CO * CI * 2;
    static constexpr uint32_t W_BYTES = KS * KS * B_TAP;
    static constexpr int TCOLS = 2 * CO <= 32 ? 32 : (2 * CO <= 64 ? 64 : (2 * CO <= 128 ? 128 : 256));
    // input-tile buffers: three (two tiles in flight while one is computed) where
    // they fit in 72 KB with the weights, else two
    static constexpr int NBUF = W_BYTES + 3 * A_BYTES <= 72 * 1024 ? 3 : 2;
    static constexpr size_t SMEM = W_BYTES + NBUF * A_BYTES;
    static_assert(CI % 16 == 0 && CO % 16 == 0 && CO <= 256, "tcgen05 shape");
};

constexpr long long TC_WAIT_LIMIT = 1ll << 26;    // mbarrier polls before a tile is declared lost

template <int CI, int CO, int KS, int INMODE, int OUTMODE, int CU>
__global__ void __launch_bounds__(CONV_THREADS)
conv_tc(ConvIn in, Bal bal, const bf16* __restrict__ W, ConvOut out, Lv lv, const int* skip, int* err) {
    using S = TcShape<CI, CO, KS>;
    constexpr uint32_t IDESC = tc_idesc(128, CO);
    extern __shared__ __align__(16) unsigned char sm[];    // no-swizzle operands need 16-byte alignment
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) unsigned long long mbar[2];
    const int H = lv.H, Wd = lv.Wd;
    const int ntx = (Wd + CONV_TW - 1) / CONV_TW, nty = (H + CONV_TH - 1) / CONV_TH;
    const int ntiles = ntx * nty;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ws = smem_u32(sm);
    const uint32_t xs0 = ws + S::W_BYTES;
    const uint32_t mb[2] = {smem_u32(&mbar[0]), smem_u32(&mbar[1])};
    // weights into K-major core matrices: (tap, co, 8 channels v) -> tap*B_TAP + (co/8)*B_SBO + v*128 + (co%8)*16;
    // issued before the wait for the previous layer (they do not depend on it)
    for (int idx = threadIdx.x; idx < KS * KS * CO * S::C8; idx += blockDim.x) {
        const int row = idx / S::C8, v = idx - row * S::C8;
        const int tap = row / CO, co = row - tap * CO;
        cp_async16(ws + (uint32_t)(tap * S::B_TAP + (co >> 3) * S::B_SBO + v * S::B_LBO + (co & 7) * 16),
                   W + (size_t)row * CI + v * 8, 16);
    }
    net_pdl_wait();
    if (skip != nullptr && *skip) {
        cp_async_commit();           // the weight copies must be part of a group for the wait to cover them
        cp_async_wait<0>();
        return;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)S::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb[0]), "r"(1u) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb[1]), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the first NBUF - 1 tiles of this CTA, one commit group each
#pragma unroll
    for (int q = 0; q < S::NBUF - 1; ++q) {
        const int t = tile + q * gridDim.x;
        if (t < ntiles)
            stage_tile<CI, S::IH, S::IW, 0, INMODE, CU, 1>(in, bal, lv, (t / ntx) * CONV_TH, (t % ntx) * CONV_TW,
                                                           S::HP, xs0 + q * S::A_BYTES);
        cp_async_commit();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    uint32_t parity[2] = {0u, 0u};
    int failed = 0;
    int buf = 0;       // accumulator (and mbarrier) of this tile: alternates
    int xb = 0;        // input buffer of this tile: cycles through NBUF
    // epilogue split: warps w and w + 4 share TMEM lanes 32 (w % 4) .. +31, each takes half the columns
    const int lanebase = (warp & 3) * 32;
    const int m = lanebase + lane;                       // GEMM row = pixel (m / 8, m % 8) of the tile
    const int cbeg = (warp >> 2) * (CO / 2);
    for (; tile < ntiles; tile += gridDim.x, buf ^= 1, xb = xb + 1 == S::NBUF ? 0 : xb + 1) {
        cp_async_wait<S::NBUF - 2>();        // this tile's group is complete; later ones may be in flight
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // staged data -> tensor-core reads
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const uint32_t xs = xs0 + xb * S::A_BYTES;
        if (threadIdx.x == 0) {
            uint32_t acc = 0u;
#pragma unroll
            for (int tap = 0; tap < KS * KS; ++tap) {
                const int ky = tap / KS, kx = tap - ky * KS;
#pragma unroll
                for (int kc = 0; kc < CI / 16; ++kc) {
                    const uint64_t ad = tc_sdesc(xs + ky * S::A_SBO + 2 * kc * S::A_LBO + kx * 16, S::A_LBO, S::A_SBO);
                    const uint64_t bd = tc_sdesc(ws + tap * S::B_TAP + 2 * kc * S::B_LBO, S::B_LBO, S::B_SBO);
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + buf * CO),
                        "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                        : "memory");
                    acc = 1u;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb[buf])
                         : "memory");
        }
        // the buffer of the previous tile is free (its MMAs completed before its epilogue):
        // stage the tile NBUF - 1 ahead into it
        if (tile + gridDim.x >= ntiles) net_pdl_trigger();     // last tile of this CTA: release the next layer
        const int pre = tile + (S::NBUF - 1) * gridDim.x;
        if (pre < ntiles) {
            const int pb = xb == 0 ? S::NBUF - 1 : xb - 1;
            stage_tile<CI, S::IH, S::IW, 0, INMODE, CU, 1>(in, bal, lv, (pre / ntx) * CONV_TH,
                                                           (pre % ntx) * CONV_TW, S::HP, xs0 + pb * S::A_BYTES);
        }
        cp_async_commit();
        bool ready = false;
        for (long long it = 0; it < TC_WAIT_LIMIT && !ready; ++it) ready = mbar_test(mb[buf], parity[buf]);
        parity[buf] ^= 1u;
        if (__syncthreads_or(!ready)) {
            failed = 1;
            break;
        }
        tc_fence_after();
        const int y0 = (tile / ntx) * CONV_TH, x0 = (tile % ntx) * CONV_TW;
        const int gy = y0 + (m >> 3), gx = x0 + (m & 7);
        const bool inside = gy < H && gx < Wd;
        const uint32_t taddr = tmem + ((uint32_t)lanebase << 16) + buf * CO;
        if constexpr (OUTMODE == OUT_PLANES) {
            if (warp < 4) {
                float v[8];
                tmem_ld8(taddr, v);
                if (inside) {
                    float* o = reinterpret_cast<float*>(out.o);
                    const size_t npix = (size_t)H * Wd;
#pragma unroll
                    for (int c = 0; c < MAXF; ++c) {
                        if (c >= bal.nf) break;
                        float* d = o + (size_t)c * npix + (size_t)gy * Wd + gx;
                        const float val = v[c] * bal.inv[c];
                        *d = out.accumulate ? *d + val : val;
                    }
                }
            }
        } else {
#pragma unroll
            for (int c0 = 0; c0 < CO / 2; c0 += 8) {
                float v[8];
                tmem_ld8(taddr + cbeg + c0, v);      // whole warp (collective); stores guarded below
                if (inside) {
                    const size_t base = ((size_t)gy * Wd + gx) * out.ostr + out.ooff + cbeg + c0;
                    if constexpr (OUTMODE == OUT_F32) {
                        float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(out.o) + base);
                        o[0] = make_float4(v[0], v[1], v[2], v[3]);
                        o[1] = make_float4(v[4], v[5], v[6], v[7]);
                    } else {
                        __align__(16) __nv_bfloat162 h[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                        *reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(out.o) + base) =
                            *reinterpret_cast<uint4*>(h);
                    }
                }
            }
        }
    }
    if (failed && threadIdx.x == 0 && err != nullptr) atomicExch(err, 1);
    cp_async_wait<0>();
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)S::TCOLS)
                     : "memory");
}

// dW[tap][co][ci] += sum_p dout[p][co] in[p + off(tap)][ci] over a 16x16 pixel tile.
template <int CI, int CO, int KS>
__global__ void __launch_bounds__(256)
conv_wgrad(const bf16* __restrict__ in, int istr, int ioff, const bf16* __restrict__ dout, Lv lv,
           float* __restrict__ dW) {
    constexpr int TH = 16, TW = 16, HP = KS / 2;
    constexpr int IH = TH + 2 * HP, IW = TW + 2 * HP;
    extern __shared__ __align__(16) unsigned char sm[];
    bf16* xs = reinterpret_cast<bf16*>(sm);        // [IH*IW][CI]
    bf16* ds = xs + IH * IW * CI;                  // [TH*TW][CO]
    const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
    const int H = lv.H, Wd = lv.Wd;
    const int sy0 = (y0 / lv.Hs) * lv.Hs, sy1 = min(sy0 + lv.Hs, H);   // the tile's slice
    constexpr int VPP = CI / 8;
    for (int idx = threadIdx.x; idx < IH * IW * VPP; idx += blockDim.x) {
        const int pix = idx / VPP, v = idx - pix * VPP;
        const int iy = pix / IW, ix = pix - iy * IW;
        const int gy = y0 + iy - HP, gx = x0 + ix - HP;
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if (gy >= sy0 && gy < sy1 && gx >= 0 && gx < Wd)
            val = *reinterpret_cast<const uint4*>(in + ((size_t)gy * Wd + gx) * istr + ioff + v * 8);
        *reinterpret_cast<uint4*>(xs + pix * CI + v * 8) = val;
    }
    constexpr int VPO = CO / 8;
    for (int idx = threadIdx.x; idx < TH * TW * VPO; idx += blockDim.x) {
        const int pix = idx / VPO, v = idx - pix * VPO;
        const int gy = y0 + pix / TW, gx = x0 + pix % TW;
        uint4 val = make_uint4(0u, 0u, 0u, 0u);
        if (gy < H && gx < Wd) val = *reinterpret_cast<const uint4*>(dout + ((size_t)gy * Wd + gx) * CO + v * 8);
        *reinterpret_cast<uint4*>(ds + pix * CO + v * 8) = val;
    }
    __syncthreads();
    constexpr int GROUPS = KS * KS * (CO / 4) * (CI / 4);
    for (int grp = threadIdx.x; grp < GROUPS; grp += blockDim.x) {
        const int ci4 = grp % (CI / 4), r1 = grp / (CI / 4);
        const int co4 = r1 % (CO / 4), tap = r1 / (CO / 4);
        const int dy = tap / KS - HP, dx = tap % KS - HP;
        float a[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) a[i][j] = 0.f;
        for (int p = 0; p < TH * TW; ++p) {
            const int py = p / TW, pxx = p % TW;
            const bf16* dp = ds + p * CO + co4 * 4;
            const bf16* xp = xs + ((py + HP + dy) * IW + (pxx + HP + dx)) * CI + ci4 * 4;
            float dv[4], xv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { dv[i] = __bfloat162float(dp[i]); xv[i] = __bfloat162float(xp[i]); }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) a[i][j] = fmaf(dv[i], xv[j], a[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                atomicAdd(dW + ((size_t)tap * CO + co4 * 4 + i) * CI + ci4 * 4 + j, a[i][j]);
    }
}

// ---------------------------------------------------------------- element-wise
// NHWC16 input B x from nf float32 field planes (channels nf..15 zero).
__global__ void pack_input(const float* __restrict__ x, int npix, Bal bal, bf16* __restrict__ out,
                           const int* skip) {
    if (skip != nullptr && *skip) return;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        __align__(16) bf16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c)
            v[c] = __float2bfloat16(c < MAXF && c < bal.nf ? bal.b[c] * x[(size_t)c * npix + p] : 0.f);
        reinterpret_cast<uint4*>(out + (size_t)p * 16)[0] = reinterpret_cast<uint4*>(v)[0];
        reinterpret_cast<uint4*>(out + (size_t)p * 16)[1] = reinterpret_cast<uint4*>(v)[1];
    }
}

// Coarse level of a fine level f: half the columns and slice rows, half the
// slices when d3 = 1.
__host__ __device__ __forceinline__ Lv coarser(const Lv& f) {
    return Lv{f.H / (f.d3 ? 4 : 2), f.Wd / 2, f.Hs / 2, f.d3};
}

// average pooling (2x2, or 2x2x2 when f.d3): out (coarse level) from in (fine level f), C channels.
__global__ void avgpool2(const bf16* __restrict__ in, int istr, int ioff, bf16* __restrict__ out, int ostr,
                         int ooff, int C, Lv f, const int* skip) {
    if (skip != nullptr && *skip) return;
    const Lv c_ = coarser(f);
    const int w = c_.Wd, Wd = f.Wd;
    const size_t total = (size_t)c_.H * w * C;
    const float wgt = f.d3 ? 0.125f : 0.25f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int y = (int)(q / w), x = (int)(q - (size_t)y * w);
        float s = 0.f;
        for (int dz = 0; dz <= f.d3; ++dz)
#pragma unroll
            for (int d = 0; d < 4; ++d)
                s += __bfloat162float(in[((size_t)fine_row(y, dz, d / 2, f) * Wd + 2 * x + d % 2) * istr + ioff + c]);
        out[q * ostr + ooff + c] = __float2bfloat16(wgt * s);
    }
}

// nearest upsampling x2 (x2x2 when f.d3): out (fine level f) from in (its coarse level), C channels.
__global__ void upsample2(const bf16* __restrict__ in, int istr, int ioff, bf16* __restrict__ out, int ostr,
                          int ooff, int C, Lv f, const int* skip) {
    if (skip != nullptr && *skip) return;
    const int Wd = f.Wd;
    const size_t total = (size_t)f.H * Wd * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t p = i / C;
        const int y = (int)(p / Wd), x = (int)(p - (size_t)y * Wd);
        out[p * ostr + ooff + c] = in[((size_t)coarse_row(y, f) * (Wd / 2) + x / 2) * istr + ioff + c];
    }
}

// backward of nearest upsampling: out (coarse level of f) = sums over the children of in (fine level f).
__global__ void upsample2_bwd(const bf16* __restrict__ in, int istr, int ioff, bf16* __restrict__ out, int C,
                              Lv f) {
    const Lv c_ = coarser(f);
    const int w = c_.Wd, Wd = f.Wd;
    const size_t total = (size_t)c_.H * w * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int y = (int)(q / w), x = (int)(q - (size_t)y * w);
        float s = 0.f;
        for (int dz = 0; dz <= f.d3; ++dz)
#pragma unroll
            for (int d = 0; d < 4; ++d)
                s += __bfloat162float(in[((size_t)fine_row(y, dz, d / 2, f) * Wd + 2 * x + d % 2) * istr + ioff + c]);
        out[q * C + c] = __float2bfloat16(s);
    }
}

// gradient of a skip that feeds both a concat slot and an average pool:
// out (fine level f, C) = dcat[.., off:off+C] + w up(dsmall), w = 1/4 (1/8 when f.d3)
__global__ void skip_grad(const bf16* __restrict__ dcat, int cstr, int coff, const bf16* __restrict__ dsmall,
                          bf16* __restrict__ out, int C, Lv f) {
    const int Wd = f.Wd;
    const size_t total = (size_t)f.H * Wd * C;
    const float wgt = f.d3 ? 0.125f : 0.25f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t p = i / C;
        const int y = (int)(p / Wd), x = (int)(p - (size_t)y * Wd);
        const float v = __bfloat162float(dcat[p * cstr + coff + c]) +
                        wgt * __bfloat162float(dsmall[((size_t)coarse_row(y, f) * (Wd / 2) + x / 2) * C + c]);
        out[p * C + c] = __float2bfloat16(v);
    }
}

// out += ||B x||^2 over the nf field planes
__global__ void sumsq(const float* __restrict__ x, int npix, Bal bal, double* out) {
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)bal.nf * npix;
         i += (size_t)gridDim.x * blockDim.x) {
        const double v = (double)(bal.b[i / npix] * x[i]);
        s += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// With y the raw output (balanced units): dy = (y - B t) / ||B x||^2
// (channels 0..nf-1), loss += 1/2 (y - B t)^2 / ||B x||^2.
__global__ void loss_grad(const float* __restrict__ y, const float* __restrict__ t, int npix, Bal bal,
                          const double* xn2, bf16* __restrict__ dy, double* loss) {
    const float inv = (float)(1.0 / fmax(*xn2, 1e-300));
    double s = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        __align__(16) bf16 v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            float d = 0.f;
            if (c < MAXF && c < bal.nf) {
                d = y[(size_t)p * 16 + c] - bal.b[c] * t[(size_t)c * npix + p];
                s += 0.5 * (double)d * (double)d;
            }
            v[c] = __float2bfloat16(d * inv);
        }
        reinterpret_cast<uint4*>(dy + (size_t)p * 16)[0] = reinterpret_cast<uint4*>(v)[0];
        reinterpret_cast<uint4*>(dy + (size_t)p * 16)[1] = reinterpret_cast<uint4*>(v)[1];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * (double)inv);
}

// Wt[tap'][ci][co] = W[KS*KS-1-tap'][co][ci]  (weights of the input-gradient convolution)
__global__ void flip_transpose(const bf16* __restrict__ W, bf16* __restrict__ Wt, int CI, int CO, int KK) {
    const int total = KK * CI * CO;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int co = i % CO, r = i / CO;
        const int ci = r % CI, tp = r / CI;
        Wt[i] = W[((size_t)(KK - 1 - tp) * CO + co) * CI + ci];
    }
}

__global__ void adam_step(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, bf16* __restrict__ wb, size_t n, float lr, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
        w[i] = wi;
        wb[i] = __float2bfloat16(wi);
    }
}

// wc[tap][co][ci] = sum_m W0d[co][m] W0c[tap][m][ci] (float32 sums, rounded once), rows co >= nf zero:
// the 1x1 layer L0d applied after L0c, as one 3x3 48 -> 16 layer.
__global__ void compose_l0(const float* __restrict__ w0c, const float* __restrict__ w0d, int nf,
                           bf16* __restrict__ wc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 9 * 16 * 48; i += gridDim.x * blockDim.x) {
        const int ci = i % 48, r = i / 48;
        const int co = r % 16, tap = r / 16;
        float acc = 0.f;
        if (co < nf)
            for (int m = 0; m < 16; ++m) acc = fmaf(w0d[co * 16 + m], w0c[((size_t)tap * 16 + m) * 48 + ci], acc);
        wc[i] = __float2bfloat16(acc);
    }
}

__global__ void to_bf16(const float* __restrict__ w, bf16* __restrict__ wb, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16(w[i]);
}

int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b > 1216 ? 1216 : (b > 0 ? b : 1));
}

// Convolution engines: tcgen05.mma (conv_tc, the default) or the legacy
// mma.sync path (conv_mma); both compute the same layer.
enum { ENGINE_TCGEN05 = 0, ENGINE_MMA_SYNC = 1 };

template <int CI, int CO, int KS, int INMODE, int OUTMODE, int CU = 0>
cudaError_t conv_ex_tc(const ConvIn& in, const Bal& bal, const bf16* W, const ConvOut& out, const Lv& lv,
                       cudaStream_t s, const int* skip, int* err) {
    using S = TcShape<CI, CO, KS>;
    auto kern = conv_tc<CI, CO, KS, INMODE, OUTMODE, CU>;
    static int max_ctas = 0;   // resident CTAs on the device (persistent grid)
    if (max_ctas == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
            return e;
        int dev = 0, sms = 0, regs_sm = 0, smem_sm = 0, thr_sm = 0, smem_res = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess)
            return e;
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        // The runtime's occupancy calculator reports one CTA per SM for any kernel
        // that allocates tensor memory; the SM holds as many as its registers,
        // threads and shared memory allow, and tcgen05.alloc waits only when the
        // 512 TMEM columns are taken, so the grid is sized from those limits and
        // from 512 / TCOLS.
        const int regs_cta = ((fa.numRegs + 7) / 8 * 8) * CONV_THREADS;
        int per_sm = regs_cta > 0 ? regs_sm / regs_cta : 1;
        per_sm = std::min(per_sm, thr_sm / CONV_THREADS);
        per_sm = std::min(per_sm, smem_sm / (int)(S::SMEM + fa.sharedSizeBytes + smem_res));
        per_sm = std::min(per_sm, 512 / S::TCOLS);
        max_ctas = sms * std::max(per_sm, 1);
    }
    const int ntiles = ((lv.Wd + CONV_TW - 1) / CONV_TW) * ((lv.H + CONV_TH - 1) / CONV_TH);
    const int grid = ntiles < max_ctas ? ntiles : max_ctas;
    return net_launch(kern, grid, CONV_THREADS, S::SMEM, s, in, bal, W, out, lv, skip, err);
}

template <int CI, int CO, int KS, int INMODE, int OUTMODE, int CU = 0>
cudaError_t conv_ex(const ConvIn& in, const Bal& bal, const bf16* W, const ConvOut& out, const Lv& lv,
                    cudaStream_t s, const int* skip, int engine = ENGINE_TCGEN05, int* err = nullptr) {
    if (engine == ENGINE_TCGEN05) return conv_ex_tc<CI, CO, KS, INMODE, OUTMODE, CU>(in, bal, W, out, lv, s, skip, err);
    using S = ConvShape<CI, CO, KS>;
    auto kern = conv_mma<CI, CO, KS, INMODE, OUTMODE, CU>;
    static int max_ctas = 0;   // resident CTAs on the device (persistent grid)
    if (max_ctas == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CONV_THREADS, S::SMEM)) != cudaSuccess)
            return e;
        max_ctas = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int ntiles = ((lv.Wd + CONV_TW - 1) / CONV_TW) * ((lv.H + CONV_TH - 1) / CONV_TH);
    const int grid = ntiles < max_ctas ? ntiles : max_ctas;
    return net_launch(kern, grid, CONV_THREADS, S::SMEM, s, in, bal, W, out, lv, skip);
}

// plain NHWC -> NHWC convolution (training path)
template <int CI, int CO, int KS, bool OUTF32>
cudaError_t conv(const bf16* in, int istr, int ioff, const bf16* W, void* out, int ostr, int ooff, const Lv& lv,
                 cudaStream_t s, const int* skip, int engine, int* err) {
    ConvIn ci{in, istr, ioff, nullptr, 0, 0, nullptr};
    ConvOut co{out, ostr, ooff, 0};
    Bal bal{};
    return conv_ex<CI, CO, KS, IN_NHWC, OUTF32 ? OUT_F32 : OUT_BF16>(ci, bal, W, co, lv, s, skip, engine, err);
}

template <int CI, int CO, int KS>
cudaError_t wgrad(const bf16* in, int istr, int ioff, const bf16* dout, const Lv& lv, float* dW, cudaStream_t s) {
    constexpr int HP = KS / 2;
    const size_t sm = sizeof(bf16) * ((16 + 2 * HP) * (16 + 2 * HP) * CI + 256 * CO);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(conv_wgrad<CI, CO, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((lv.Wd + 15) / 16, (lv.H + 15) / 16);
    conv_wgrad<CI, CO, KS><<<grid, 256, sm, s>>>(in, istr, ioff, dout, lv, dW);
    return cudaGetLastError();
}

uint64_t splitmix(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct UNet {
    int nx, ny, nz, dim;
    Lv lv[3];                               // levels 0 (the grid), 1, 2
    size_t npix;                            // points of the grid
    size_t nw;
    size_t woff[NL + 1];
    float *w32, *g32, *m32, *v32;           // master weights, gradient, Adam moments
    bf16 *wb, *wt;                          // bfloat16 weights, flipped/transposed copies
    bf16* wc;                               // L0d composed with L0c (inference), [tap][16][48]
    bool wc_stale;                          // the composition predates the current weights
    unsigned long long version;             // bumped whenever what an apply computes may change
    // activations (NHWC bfloat16) and gradients
    bf16 *x0, *h0a, *cat0, *p1, *h1a, *cat1, *p2, *h2a, *h2b, *h1c, *h0c;
    bf16 *dy, *dh0c, *dcat0, *dh1c, *dcat1, *dh2b, *dh2a, *dp2, *ds1, *dh1a, *dp1, *ds0, *dh0a;
    float* yf;                              // output NHWC16 float32
    double* scal;                           // [0] ||B x||^2, [1] loss
    int* derr;                              // set by a convolution whose tensor-core wait timed out
    int engine;                             // ENGINE_TCGEN05 or ENGINE_MMA_SYNC
    int step;
    Bal bal;
};

static void free_net(UNet* n) {
    void* p[] = {n->w32, n->g32, n->m32, n->v32, n->wb, n->wt, n->wc, n->x0, n->h0a, n->cat0, n->p1, n->h1a, n->cat1,
                 n->p2, n->h2a, n->h2b, n->h1c, n->h0c, n->dy, n->dh0c, n->dcat0, n->dh1c, n->dcat1, n->dh2b,
                 n->dh2a, n->dp2, n->ds1, n->dh1a, n->dp1, n->ds0, n->dh0a, n->yf, n->scal, n->derr};
    for (void* q : p)
        if (q) cudaFree(q);
}

bool unet_grid_ok(int dim, int nx, int ny, int nz) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || nx % 32) return false;
    if (dim == 2) return ny == 1 && nz % 32 == 0;
    // slices of ny rows hold whole 16-row tiles at every level; z pools twice
    return dim == 3 && ny % 64 == 0 && nz % 4 == 0 && (long long)nx * ny * nz < (1ll << 31);
}

// Versions are unique over the process (a new network never repeats an old one's).
static unsigned long long next_version() {
    static std::atomic<unsigned long long> counter{0};
    return ++counter;
}

UNet* unet_create(int dim, int nx, int ny, int nz, const double* balance, unsigned long long seed,
                  cudaError_t* err) {
    *err = cudaSuccess;
    if (!unet_grid_ok(dim, nx, ny, nz)) { *err = cudaErrorInvalidValue; return nullptr; }
    const int nf = dim == 2 ? 4 : 5;
    for (int f = 0; f < nf; ++f)
        if (!(balance[f] > 0.0) || !isfinite(balance[f])) { *err = cudaErrorInvalidValue; return nullptr; }
    UNet* n = new (std::nothrow) UNet;
    if (!n) { *err = cudaErrorMemoryAllocation; return nullptr; }
    memset(n, 0, sizeof(*n));
    n->version = next_version();
    n->nx = nx;
    n->ny = ny;
    n->nz = nz;
    n->dim = dim;
    n->lv[0] = dim == 2 ? Lv{nz, nx, nz, 0} : Lv{nz * ny, nx, ny, 1};
    n->lv[1] = coarser(n->lv[0]);
    n->lv[2] = coarser(n->lv[1]);
    n->npix = (size_t)nx * ny * nz;
    n->bal.nf = nf;
    for (int f = 0; f < MAXF; ++f) {
        n->bal.b[f] = f < nf ? (float)balance[f] : 0.f;
        n->bal.inv[f] = f < nf ? (float)(1.0 / balance[f]) : 0.f;
    }
    size_t o = 0;
    for (int l = 0; l < NL; ++l) { n->woff[l] = o; o += (size_t)KSZ[l] * KSZ[l] * COUT[l] * CIN[l]; }
    n->woff[NL] = o;
    n->nw = o;
    const size_t P0 = n->npix, P1 = (size_t)n->lv[1].H * n->lv[1].Wd, P2 = (size_t)n->lv[2].H * n->lv[2].Wd;
    auto A = [&](void** p, size_t bytes) {
        if (*err == cudaSuccess) *err = cudaMalloc(p, bytes);
    };
    A((void**)&n->w32, o * 4); A((void**)&n->g32, o * 4); A((void**)&n->m32, o * 4); A((void**)&n->v32, o * 4);
    A((void**)&n->wb, o * 2); A((void**)&n->wt, o * 2);
    A((void**)&n->wc, (size_t)9 * 16 * 48 * 2);
    A((void**)&n->x0, P0 * 16 * 2); A((void**)&n->h0a, P0 * 16 * 2); A((void**)&n->cat0, P0 * 48 * 2);
    A((void**)&n->p1, P1 * 16 * 2); A((void**)&n->h1a, P1 * 32 * 2); A((void**)&n->cat1, P1 * 96 * 2);
    A((void**)&n->p2, P2 * 32 * 2); A((void**)&n->h2a, P2 * 64 * 2); A((void**)&n->h2b, P2 * 64 * 2);
    A((void**)&n->h1c, P1 * 32 * 2); A((void**)&n->h0c, P0 * 16 * 2);
    A((void**)&n->dy, P0 * 16 * 2); A((void**)&n->dh0c, P0 * 16 * 2); A((void**)&n->dcat0, P0 * 48 * 2);
    A((void**)&n->dh1c, P1 * 32 * 2); A((void**)&n->dcat1, P1 * 96 * 2); A((void**)&n->dh2b, P2 * 64 * 2);
    A((void**)&n->dh2a, P2 * 64 * 2); A((void**)&n->dp2, P2 * 32 * 2); A((void**)&n->ds1, P1 * 32 * 2);
    A((void**)&n->dh1a, P1 * 32 * 2); A((void**)&n->dp1, P1 * 16 * 2); A((void**)&n->ds0, P0 * 16 * 2);
    A((void**)&n->dh0a, P0 * 16 * 2); A((void**)&n->yf, P0 * 16 * 4); A((void**)&n->scal, 16 * 8);
    A((void**)&n->derr, sizeof(int));
    if (*err == cudaSuccess) *err = cudaMemset(n->derr, 0, sizeof(int));
    n->engine = ENGINE_TCGEN05;
    if (*err != cudaSuccess) { free_net(n); delete n; return nullptr; }
    // seeded init: N(0, 1/fan_in) on real input channels; the last layer and the
    // padded input / output channels start at zero (untrained net = zero map)
    std::vector<float> w(o, 0.f);
    uint64_t st = seed;
    for (int l = 0; l < NL; ++l) {
        if (l == L0d) continue;
        const int ci_real = l == L0a ? nf : CIN[l];
        const float sd = sqrtf(1.0f / (KSZ[l] * KSZ[l] * ci_real));
        for (int tp = 0; tp < KSZ[l] * KSZ[l]; ++tp)
            for (int co = 0; co < COUT[l]; ++co)
                for (int ci = 0; ci < ci_real; ++ci) {
                    const double u1 = ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
                    const double u2 = ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
                    const double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
                    w[n->woff[l] + ((size_t)tp * COUT[l] + co) * CIN[l] + ci] = (float)(sd * z);
                }
    }
    *err = unet_set_weights(n, w.data(), 0);
    if (*err == cudaSuccess) *err = cudaStreamSynchronize(0);
    if (*err != cudaSuccess) { free_net(n); delete n; return nullptr; }
    return n;
}

void unet_destroy(UNet* n) {
    if (!n) return;
    free_net(n);
    delete n;
}

size_t unet_num_weights(const UNet* n) { return n->nw; }

cudaError_t unet_get_weights(UNet* n, float* host, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(host, n->w32, n->nw * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t unet_set_weights(UNet* n, const float* host, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(n->w32, host, n->nw * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    to_bf16<<<grid_for(n->nw), 256, 0, s>>>(n->w32, n->wb, n->nw);
    n->wc_stale = true;
    n->version = next_version();
    if ((e = cudaMemsetAsync(n->m32, 0, n->nw * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(n->v32, 0, n->nw * 4, s)) != cudaSuccess) return e;
    n->step = 0;
    return cudaGetLastError();
}

#define UCK(x)                              \
    do {                                    \
        cudaError_t e_ = (x);               \
        if (e_ != cudaSuccess) return e_;   \
    } while (0)

static cudaError_t forward(UNet* n, const float* x, cudaStream_t s, const int* skip) {
    const Lv L0 = n->lv[0], L1 = n->lv[1], L2 = n->lv[2];
    const size_t P0 = n->npix, P1 = (size_t)L1.H * L1.Wd, P2 = (size_t)L2.H * L2.Wd;
    const bf16* w = n->wb;
    pack_input<<<grid_for(P0), 256, 0, s>>>(x, (int)P0, n->bal, n->x0, skip);
    UCK((conv<16, 16, 3, false>(n->x0, 16, 0, w + n->woff[L0a], n->h0a, 16, 0, L0, s, skip, n->engine, n->derr)));
    UCK((conv<16, 16, 3, false>(n->h0a, 16, 0, w + n->woff[L0b], n->cat0, 48, 32, L0, s, skip, n->engine, n->derr)));
    avgpool2<<<grid_for(P1 * 16), 256, 0, s>>>(n->cat0, 48, 32, n->p1, 16, 0, 16, L0, skip);
    UCK((conv<16, 32, 3, false>(n->p1, 16, 0, w + n->woff[L1a], n->h1a, 32, 0, L1, s, skip, n->engine, n->derr)));
    UCK((conv<32, 32, 3, false>(n->h1a, 32, 0, w + n->woff[L1b], n->cat1, 96, 64, L1, s, skip, n->engine, n->derr)));
    avgpool2<<<grid_for(P2 * 32), 256, 0, s>>>(n->cat1, 96, 64, n->p2, 32, 0, 32, L1, skip);
    UCK((conv<32, 64, 3, false>(n->p2, 32, 0, w + n->woff[L2a], n->h2a, 64, 0, L2, s, skip, n->engine, n->derr)));
    UCK((conv<64, 64, 3, false>(n->h2a, 64, 0, w + n->woff[L2b], n->h2b, 64, 0, L2, s, skip, n->engine, n->derr)));
    upsample2<<<grid_for(P1 * 64), 256, 0, s>>>(n->h2b, 64, 0, n->cat1, 96, 0, 64, L1, skip);
    UCK((conv<96, 32, 3, false>(n->cat1, 96, 0, w + n->woff[L1c], n->h1c, 32, 0, L1, s, skip, n->engine, n->derr)));
    upsample2<<<grid_for(P0 * 32), 256, 0, s>>>(n->h1c, 32, 0, n->cat0, 48, 0, 32, L0, skip);
    UCK((conv<48, 16, 3, false>(n->cat0, 48, 0, w + n->woff[L0c], n->h0c, 16, 0, L0, s, skip, n->engine, n->derr)));
    UCK((conv<16, 16, 1, true>(n->h0c, 16, 0, w + n->woff[L0d], n->yf, 16, 0, L0, s, skip, n->engine, n->derr)));
    return cudaGetLastError();
}

// Inference forward with pooling, upsampling + concatenation, input packing
// and output unpacking fused into the convolutions, and L0d composed into
// L0c (8 launches; forward() computes the same map layer by layer, rounding
// the L0c output to bfloat16 where this one rounds the composed weights).
static cudaError_t forward_fused(UNet* n, const float* x, float* y, int accumulate, cudaStream_t s,
                                 const int* skip) {
    const Lv L0 = n->lv[0], L1 = n->lv[1], L2 = n->lv[2];
    const bf16* w = n->wb;
    const ConvIn none{nullptr, 0, 0, nullptr, 0, 0, nullptr};
    auto nhwc = [&](const bf16* a, int str, int off) { ConvIn c = none; c.a = a; c.astr = str; c.aoff = off; return c; };
    auto to = [&](void* o, int str, int off) { return ConvOut{o, str, off, 0}; };
    ConvIn pk = none;
    pk.x = x;
    UCK((conv_ex<16, 16, 3, IN_PACK, OUT_BF16>(pk, n->bal, w + n->woff[L0a], to(n->h0a, 16, 0), L0, s, skip, n->engine, n->derr)));
    UCK((conv_ex<16, 16, 3, IN_NHWC, OUT_BF16>(nhwc(n->h0a, 16, 0), n->bal, w + n->woff[L0b], to(n->cat0, 48, 32), L0, s, skip, n->engine, n->derr)));
    UCK((conv_ex<16, 32, 3, IN_POOL, OUT_BF16>(nhwc(n->cat0, 48, 32), n->bal, w + n->woff[L1a], to(n->h1a, 32, 0), L1, s, skip, n->engine, n->derr)));
    UCK((conv_ex<32, 32, 3, IN_NHWC, OUT_BF16>(nhwc(n->h1a, 32, 0), n->bal, w + n->woff[L1b], to(n->cat1, 96, 64), L1, s, skip, n->engine, n->derr)));
    UCK((conv_ex<32, 64, 3, IN_POOL, OUT_BF16>(nhwc(n->cat1, 96, 64), n->bal, w + n->woff[L2a], to(n->h2a, 64, 0), L2, s, skip, n->engine, n->derr)));
    UCK((conv_ex<64, 64, 3, IN_NHWC, OUT_BF16>(nhwc(n->h2a, 64, 0), n->bal, w + n->woff[L2b], to(n->h2b, 64, 0), L2, s, skip, n->engine, n->derr)));
    ConvIn uc1{n->h2b, 64, 0, n->cat1, 96, 64, nullptr};
    UCK((conv_ex<96, 32, 3, IN_UPCAT, OUT_BF16, 64>(uc1, n->bal, w + n->woff[L1c], to(n->h1c, 32, 0), L1, s,
                                                    skip, n->engine, n->derr)));
    // L0c and the 1x1 L0d are one linear map: the composed 3x3 48 -> 16 layer writes the field planes
    ConvIn uc0{n->h1c, 32, 0, n->cat0, 48, 32, nullptr};
    ConvOut pl{y, 0, 0, accumulate};
    UCK((conv_ex<48, 16, 3, IN_UPCAT, OUT_PLANES, 32>(uc0, n->bal, n->wc, pl, L0, s,
                                                    skip, n->engine, n->derr)));
    return cudaGetLastError();
}

// transposed weights of layer l into wt (same offsets)
static cudaError_t transpose_w(UNet* n, int l, cudaStream_t s) {
    const int kk = KSZ[l] * KSZ[l];
    flip_transpose<<<grid_for((size_t)kk * CIN[l] * COUT[l]), 256, 0, s>>>(n->wb + n->woff[l], n->wt + n->woff[l],
                                                                           CIN[l], COUT[l], kk);
    return cudaGetLastError();
}

static cudaError_t backward(UNet* n, cudaStream_t s) {
    const Lv L0 = n->lv[0], L1 = n->lv[1], L2 = n->lv[2];
    const size_t P0 = n->npix, P1 = (size_t)L1.H * L1.Wd, P2 = (size_t)L2.H * L2.Wd;
    float* g = n->g32;
    const bf16* wt = n->wt;
    UCK(cudaMemsetAsync(g, 0, n->nw * 4, s));
    for (int l = 0; l < NL; ++l) UCK(transpose_w(n, l, s));
    UCK((wgrad<16, 16, 1>(n->h0c, 16, 0, n->dy, L0, g + n->woff[L0d], s)));
    UCK((conv<16, 16, 1, false>(n->dy, 16, 0, wt + n->woff[L0d], n->dh0c, 16, 0, L0, s, nullptr, n->engine, n->derr)));
    UCK((wgrad<48, 16, 3>(n->cat0, 48, 0, n->dh0c, L0, g + n->woff[L0c], s)));
    UCK((conv<16, 48, 3, false>(n->dh0c, 16, 0, wt + n->woff[L0c], n->dcat0, 48, 0, L0, s, nullptr, n->engine, n->derr)));
    upsample2_bwd<<<grid_for(P1 * 32), 256, 0, s>>>(n->dcat0, 48, 0, n->dh1c, 32, L0);
    UCK((wgrad<96, 32, 3>(n->cat1, 96, 0, n->dh1c, L1, g + n->woff[L1c], s)));
    UCK((conv<32, 96, 3, false>(n->dh1c, 32, 0, wt + n->woff[L1c], n->dcat1, 96, 0, L1, s, nullptr, n->engine, n->derr)));
    upsample2_bwd<<<grid_for(P2 * 64), 256, 0, s>>>(n->dcat1, 96, 0, n->dh2b, 64, L1);
    UCK((wgrad<64, 64, 3>(n->h2a, 64, 0, n->dh2b, L2, g + n->woff[L2b], s)));
    UCK((conv<64, 64, 3, false>(n->dh2b, 64, 0, wt + n->woff[L2b], n->dh2a, 64, 0, L2, s, nullptr, n->engine, n->derr)));
    UCK((wgrad<32, 64, 3>(n->p2, 32, 0, n->dh2a, L2, g + n->woff[L2a], s)));
    UCK((conv<64, 32, 3, false>(n->dh2a, 64, 0, wt + n->woff[L2a], n->dp2, 32, 0, L2, s, nullptr, n->engine, n->derr)));
    skip_grad<<<grid_for(P1 * 32), 256, 0, s>>>(n->dcat1, 96, 64, n->dp2, n->ds1, 32, L1);
    UCK((wgrad<32, 32, 3>(n->h1a, 32, 0, n->ds1, L1, g + n->woff[L1b], s)));
    UCK((conv<32, 32, 3, false>(n->ds1, 32, 0, wt + n->woff[L1b], n->dh1a, 32, 0, L1, s, nullptr, n->engine, n->derr)));
    UCK((wgrad<16, 32, 3>(n->p1, 16, 0, n->dh1a, L1, g + n->woff[L1a], s)));
    UCK((conv<32, 16, 3, false>(n->dh1a, 32, 0, wt + n->woff[L1a], n->dp1, 16, 0, L1, s, nullptr, n->engine, n->derr)));
    skip_grad<<<grid_for(P0 * 16), 256, 0, s>>>(n->dcat0, 48, 32, n->dp1, n->ds0, 16, L0);
    UCK((wgrad<16, 16, 3>(n->h0a, 16, 0, n->ds0, L0, g + n->woff[L0b], s)));
    UCK((conv<16, 16, 3, false>(n->ds0, 16, 0, wt + n->woff[L0b], n->dh0a, 16, 0, L0, s, nullptr, n->engine, n->derr)));
    UCK((wgrad<16, 16, 3>(n->x0, 16, 0, n->dh0a, L0, g + n->woff[L0a], s)));
    return cudaGetLastError();
}

cudaError_t unet_set_engine(UNet* n, int engine) {
    if (engine != ENGINE_TCGEN05 && engine != ENGINE_MMA_SYNC) return cudaErrorInvalidValue;
    n->engine = engine;
    n->version = next_version();
    return cudaSuccess;
}

int unet_engine(const UNet* n) { return n->engine; }

cudaError_t unet_check(UNet* n, cudaStream_t s) {
    int e = 0;
    UCK(cudaMemcpyAsync(&e, n->derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    UCK(cudaStreamSynchronize(s));
    return e ? cudaErrorLaunchTimeout : cudaSuccess;
}

cudaError_t unet_prepare(UNet* n, cudaStream_t s) {
    if (n->wc_stale) {
        compose_l0<<<27, 256, 0, s>>>(n->w32 + n->woff[L0c], n->w32 + n->woff[L0d], n->bal.nf, n->wc);
        UCK(cudaGetLastError());
        n->wc_stale = false;
    }
    return cudaSuccess;
}

unsigned long long unet_version(const UNet* n) { return n->version; }

cudaError_t unet_apply(UNet* n, const float* x, float* y, int accumulate, const int* skip, cudaStream_t s) {
    UCK(unet_prepare(n, s));
    return forward_fused(n, x, y, accumulate, s, skip);
}

int unet_launches_per_apply() { return 8; }

static cudaError_t loss_and_dy(UNet* n, const float* x, const float* t, cudaStream_t s) {
    const int npix = (int)n->npix;
    UCK(cudaMemsetAsync(n->scal, 0, 2 * sizeof(double), s));
    sumsq<<<grid_for((size_t)n->bal.nf * npix), 256, 0, s>>>(x, npix, n->bal, n->scal);
    loss_grad<<<grid_for(npix), 256, 0, s>>>(n->yf, t, npix, n->bal, n->scal, n->dy, n->scal + 1);
    return cudaGetLastError();
}

cudaError_t unet_loss_grad(UNet* n, const float* x, const float* t, double* loss, float* grads_host,
                           cudaStream_t s) {
    UCK(forward(n, x, s, nullptr));
    UCK(loss_and_dy(n, x, t, s));
    if (grads_host) UCK(backward(n, s));
    double sc[2];
    UCK(cudaMemcpyAsync(sc, n->scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
    if (grads_host) UCK(cudaMemcpyAsync(grads_host, n->g32, n->nw * 4, cudaMemcpyDeviceToHost, s));
    UCK(cudaStreamSynchronize(s));
    if (loss) *loss = sc[1];
    return unet_check(n, s);
}

cudaError_t unet_train(UNet* n, const float* X, const float* T, int npairs, int epochs, float lr,
                       double* loss_hist, cudaStream_t s) {
    const size_t plane = (size_t)n->bal.nf * n->npix;
    for (int ep = 0; ep < epochs; ++ep) {
        double tot = 0.0;
        for (int q = 0; q < npairs; ++q) {
            const int i = (int)((q * 7919ull + ep * 104729ull) % (unsigned long long)npairs);   // fixed shuffle
            UCK(forward(n, X + i * plane, s, nullptr));
            UCK(loss_and_dy(n, X + i * plane, T + i * plane, s));
            UCK(backward(n, s));
            n->step += 1;
            const float c1 = 1.0f / (1.0f - powf(0.9f, (float)n->step));
            const float c2 = 1.0f / (1.0f - powf(0.999f, (float)n->step));
            adam_step<<<grid_for(n->nw), 256, 0, s>>>(n->w32, n->g32, n->m32, n->v32, n->wb, n->nw, lr, c1, c2);
            n->wc_stale = true;
            n->version = next_version();
            UCK(cudaGetLastError());
            if (loss_hist) {
                double sc[2];
                UCK(cudaMemcpyAsync(sc, n->scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
                UCK(cudaStreamSynchronize(s));
                tot += sc[1];
            }
        }
        if (loss_hist) loss_hist[ep] = tot / npairs;
    }
    UCK(cudaStreamSynchronize(s));
    return unet_check(n, s);
}

}  // namespace jfnk

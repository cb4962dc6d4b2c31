// mlp.cu -- learned membrane energy: a per-triangle MLP surrogate of the
// Neo-Hookean density on the invariants (I1, I2, I3) of C3 = diag(F^T F, 1).
// Not part of the paper; it replaces the analytic density of a membrane term
// (Sec. 7.7's Neo-Hookean) by a small network whose derivatives are taken by
// the same forward mode as every other term.
//
// Network (parameters theta, 4481 FP32 master values, used BF16-rounded):
//   u = (I - m_I) / s_I,  z1 = W1 u + b1,  a1 = silu(z1),
//   z2 = W2 a1 + b2,      a2 = silu(z2),   y = w3 . a2 + b3,
//   psi = s_psi y + m_psi;  W1 64x3, W2 64x64, silu(z) = z sigma(z).
// Each sample's value, 3 tangents along u and 6 second-order terms come from
// forward mode for the value and the tangents and one reverse contraction for
// the second-order part (forward over reverse).  The 64x64 contractions run
// on the tensor cores with BF16 inputs and FP32 accumulation, in two forms:
// k_mlp_tri_tc (the default for the per-triangle table) issues tcgen05.mma
// on 128-triangle tiles with the accumulators in tensor memory;
// warp_forward8 (sample evaluation, training, and the table when the
// mma.sync form is chosen) runs mma.sync m16n8k16, one warp per 8 samples.
// Everything elementwise is FP32.
//
// Training minimises the Sobolev loss on standardised quantities
//   L = mean (y - ty)^2 + beta mean sum_k (dy/du_k - tg_k)^2
// by reverse mode through the value + tangent forward pass; the backward
// contractions (W2^T and the weight gradient) also run on the tensor cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "device_common.cuh"

namespace adm {

namespace {

constexpr int H = 64;              // hidden width
constexpr int LDW = H + 8;         // padded row of BF16 matrices in shared memory
constexpr int NP = H * 3 + H + H * H + H + H + 1;  // 4481
constexpr int WARPS = 4;           // warps per block of the MLP kernels

struct MlpSmem {
    __nv_bfloat16 W2[H * LDW];     // [i][j]: B operand of z2 = W2 a1
    __nv_bfloat16 W2T[H * LDW];    // [j][i]: B operand of d a1 = d z2 W2
    float W1[H * 3], b1[H], b2[H], w3[H], b3, norm[8];
};

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16(x)); }

// parameters of theta into shared memory, BF16-rounded (the network's weights)
__device__ void load_params(MlpSmem &S, const float *th, const float *norm)
{
    const float *W1 = th, *b1 = W1 + H * 3, *W2 = b1 + H, *b2 = W2 + H * H, *w3 = b2 + H, *b3 = w3 + H;
    for (int k = threadIdx.x; k < H * H; k += blockDim.x) {
        const int i = k / H, j = k % H;
        const __nv_bfloat16 w = __float2bfloat16(W2[k]);
        S.W2[i * LDW + j] = w;
        S.W2T[j * LDW + i] = w;
    }
    for (int k = threadIdx.x; k < H * 3; k += blockDim.x) S.W1[k] = bf16r(W1[k]);
    for (int k = threadIdx.x; k < H; k += blockDim.x) {
        S.b1[k] = bf16r(b1[k]);
        S.b2[k] = bf16r(b2[k]);
        S.w3[k] = bf16r(w3[k]);
    }
    if (threadIdx.x == 0) S.b3 = bf16r(b3[0]);
    if (threadIdx.x < 8) S.norm[threadIdx.x] = norm[threadIdx.x];
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// acc (16 x 64, m16n8 accumulator layout, n-tile nn) += A (16 x 64) B where A
// is given as per-lane fragments a[kk][4] and B through Bt[n][k] (row stride LDW)
__device__ __forceinline__ void mma_16x64(float (&acc)[8][4], const uint32_t (&a)[4][4], const __nv_bfloat16 *Bt)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
#pragma unroll
        for (int nn = 0; nn < 8; ++nn) {
            const uint32_t b0 = *reinterpret_cast<const uint32_t *>(Bt + (nn * 8 + g) * LDW + kk * 16 + 2 * t);
            const uint32_t b1 = *reinterpret_cast<const uint32_t *>(Bt + (nn * 8 + g) * LDW + kk * 16 + 2 * t + 8);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(acc[nn][0]), "+f"(acc[nn][1]), "+f"(acc[nn][2]), "+f"(acc[nn][3])
                : "r"(a[kk][0]), "r"(a[kk][1]), "r"(a[kk][2]), "r"(a[kk][3]), "r"(b0), "r"(b1));
        }
}

__device__ __forceinline__ void zero(float (&acc)[8][4])
{
#pragma unroll
    for (int nn = 0; nn < 8; ++nn)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[nn][q] = 0.0f;
}

// A-fragment / accumulator index helpers.  Lane (g, t) owns rows g and g+8
// (samples) and, for accumulator n-tile nn, columns 8 nn + 2 t + {0, 1};
// the same (row, column) set forms the A fragments of k-tile kk = nn / 2.
// Element e = nn * 4 + q: row g + 8 (q >> 1), column 8 nn + 2 t + (q & 1).
__device__ __forceinline__ int elem_row(int e) { return ((threadIdx.x & 31) >> 2) + 8 * ((e & 3) >> 1); }
__device__ __forceinline__ int elem_col(int e) { return 8 * (e >> 2) + 2 * (threadIdx.x & 3) + (e & 1); }

// SiLU and its first two derivatives: sg = sigma(z), s = z sg,
// s1 = sg (1 + z (1 - sg)), s2 = sg (1 - sg) (2 + z (1 - 2 sg)).  The fast
// exponential and divide intrinsics suffice (about 2 ulp): the network's
// activations are rounded to BF16 before every contraction.  The correctly
// rounded reciprocal cost the per-triangle network a quarter of its time.
__device__ __forceinline__ void silu_all(float z, float &sg, float &s, float &s1, float &s2)
{
    sg = __fdividef(1.0f, 1.0f + __expf(-z));
    s = z * sg;
    s1 = sg * (1.0f + z * (1.0f - sg));
    s2 = sg * (1.0f - sg) * (2.0f + z * (1.0f - 2.0f * sg));
}

// A fragments of one channel from per-element values v[32] (element order e)
__device__ __forceinline__ void to_frag(const float (&v)[32], uint32_t (&a)[4][4])
{
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        // k-tile kk covers n-tiles 2 kk (cols 2t..) and 2 kk + 1 (cols 8 + 2t..)
        const int e0 = (2 * kk) * 4, e1 = (2 * kk + 1) * 4;
        a[kk][0] = pack_bf16(v[e0 + 0], v[e0 + 1]);  // row g,   cols 2t, 2t+1
        a[kk][1] = pack_bf16(v[e0 + 2], v[e0 + 3]);  // row g+8
        a[kk][2] = pack_bf16(v[e1 + 0], v[e1 + 1]);  // row g,   cols 2t+8, 2t+9
        a[kk][3] = pack_bf16(v[e1 + 2], v[e1 + 3]);  // row g+8
    }
}

// per-row sums across the 4 lanes of a quad (same g, t = 0..3)
__device__ __forceinline__ float quad_sum(float v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

// Forward mode through the network for 8 samples per warp.  The value and
// the 3 tangents along u are carried forward: the hidden layer runs
// transposed, z2^T = W2 a1^T, with W2 (64 x 64, row = output unit) the A
// operand from shared memory and the 4 channels of a1^T (64 units x 8
// samples) B operands built by the lanes themselves.  Lane (g, t) takes
// sample g: it evaluates layer 1 for units 16 kt + 2 t + {0, 1, 8, 9},
// exactly the rows of its B fragments, and after the contraction holds every
// channel of z2 for units 16 mt + g + {0, 8} and samples 2 t + {0, 1}.
// The 6 second-order terms split as
//   d2y/du_k du_l = sum_m w3_m [silu''(z2_m) dz2_m/du_k dz2_m/du_l
//                               + silu'(z2_m) d2z2_m/du_k du_l],
// and the second part is sum_n r_n silu''(z1_n) W1_nk W1_nl with
// r = W2^T rho, rho_m = w3_m silu'(z2_m): one reverse contraction (W2^T is
// the A operand, rho the B operand) instead of carrying 6 second-order
// channels through W2.  rho and silu''(z1) pass between lanes through the
// warp's slab ws (2 x 64 x 8 floats, [unit][sample]).  Output sums over
// units close with shuffles.
// u: standardised input of sample g = lane / 4.  y[n][c]: channel c of sample
// 2 t + n (value, dy/du_k, upper Hessian uu00, uu01, uu11, uu02, uu12, uu22),
// identical in the 8 lanes of a column t.
__device__ __forceinline__ void warp_forward8(const MlpSmem &S, const float (&u)[3], float (&y)[2][10], float *ws)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    constexpr int K2[6] = {0, 0, 1, 0, 1, 2}, L2[6] = {0, 1, 1, 2, 2, 2};
    float *s2v = ws, *rho = ws + H * 8;  // [unit][sample]
    __syncwarp();                         // the previous samples' reads of the slab are done
    // layer 1 -> B fragments of the value and the tangents: b[kt][c][0] =
    // units 16kt + 2t, +1; [1] = +8, +9; silu''(z1) of each unit to the slab
    uint32_t b[4][4][2];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[2][4];
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const int i = 16 * kt + 2 * t + 8 * h + o;
                const float w0 = S.W1[3 * i], w1 = S.W1[3 * i + 1], w2 = S.W1[3 * i + 2];
                const float z = S.b1[i] + w0 * u[0] + w1 * u[1] + w2 * u[2];
                float sg, s0, s1, s2;
                silu_all(z, sg, s0, s1, s2);
                v[o][0] = s0;
                v[o][1] = s1 * w0;
                v[o][2] = s1 * w1;
                v[o][3] = s1 * w2;
                s2v[i * 8 + g] = s2;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) b[kt][c][h] = pack_bf16(v[0][c], v[1][c]);
        }
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int c = 0; c < 10; ++c) y[n][c] = 0.0f;
#pragma unroll 1
    for (int mt = 0; mt < 4; ++mt) {
        float acc[4][4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[c][q] = 0.0f;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const __nv_bfloat16 *w = S.W2 + (16 * mt + g) * LDW + 16 * kt + 2 * t;
            const uint32_t a0 = *reinterpret_cast<const uint32_t *>(w);
            const uint32_t a1 = *reinterpret_cast<const uint32_t *>(w + 8 * LDW);
            const uint32_t a2 = *reinterpret_cast<const uint32_t *>(w + 8);
            const uint32_t a3 = *reinterpret_cast<const uint32_t *>(w + 8 * LDW + 8);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                    "{%0,%1,%2,%3};\n"
                    : "+f"(acc[c][0]), "+f"(acc[c][1]), "+f"(acc[c][2]), "+f"(acc[c][3])
                    : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b[kt][c][0]), "r"(b[kt][c][1]));
        }
        // layer 2 and the output layer for units j = 16 mt + g + 8 (q >> 1),
        // samples 2 t + (q & 1): value, tangents, the first second-order
        // part; rho of the unit to the slab
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = 16 * mt + g + 8 * (q >> 1), n = q & 1;
            float sg, s0, s1, s2;
            silu_all(acc[0][q] + S.b2[j], sg, s0, s1, s2);
            const float w = S.w3[j];
            const float d[3] = {acc[1][q], acc[2][q], acc[3][q]};
            y[n][0] += w * s0;
#pragma unroll
            for (int k = 0; k < 3; ++k) y[n][1 + k] += w * s1 * d[k];
#pragma unroll
            for (int m = 0; m < 6; ++m) y[n][4 + m] += w * s2 * d[K2[m]] * d[L2[m]];
            rho[j * 8 + 2 * t + n] = w * s1;
        }
    }
    __syncwarp();  // rho and silu''(z1) of all units and samples are in the slab
    // reverse contraction r = W2^T rho (rows: layer-1 units n = 16 nt + g +
    // 8 (q >> 1); columns: samples 2 t + (q & 1)), then the second part of
    // the second-order terms
#pragma unroll 1
    for (int nt = 0; nt < 4; ++nt) {
        float r[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const __nv_bfloat16 *w = S.W2T + (16 * nt + g) * LDW + 16 * kt + 2 * t;
            const uint32_t a0 = *reinterpret_cast<const uint32_t *>(w);
            const uint32_t a1 = *reinterpret_cast<const uint32_t *>(w + 8 * LDW);
            const uint32_t a2 = *reinterpret_cast<const uint32_t *>(w + 8);
            const uint32_t a3 = *reinterpret_cast<const uint32_t *>(w + 8 * LDW + 8);
            const int m0 = 16 * kt + 2 * t;
            const uint32_t b0 = pack_bf16(rho[m0 * 8 + g], rho[(m0 + 1) * 8 + g]);
            const uint32_t b1 = pack_bf16(rho[(m0 + 8) * 8 + g], rho[(m0 + 9) * 8 + g]);
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};\n"
                : "+f"(r[0]), "+f"(r[1]), "+f"(r[2]), "+f"(r[3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = 16 * nt + g + 8 * (q >> 1), n = q & 1;
            const float p = r[q] * s2v[i * 8 + 2 * t + n];
            const float wk[3] = {S.W1[3 * i], S.W1[3 * i + 1], S.W1[3 * i + 2]};
#pragma unroll
            for (int m = 0; m < 6; ++m) y[n][4 + m] += p * wk[K2[m]] * wk[L2[m]];
        }
    }
    // sum over the 8 lanes g of each column t
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int c = 0; c < 10; ++c) {
            float v = y[n][c];
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            y[n][c] = v + (c == 0 ? S.b3 : 0.0f);
        }
}

// network outputs of sample p (channel order of warp_forward8) in the units
// of the invariants: psi, dpsi/dI (3), upper Hessian in I (6).  Lane (g, t)
// writes channels g and g + 8 of samples 2 t + n.
__device__ __forceinline__ void store_unstandardised(const MlpSmem &S, const float (&y)[2][10], int64_t base,
                                                     int64_t n_valid, float *out)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float sp = S.norm[7];
#pragma unroll
    for (int n = 0; n < 2; ++n) {
        const int64_t p = base + 2 * t + n;
        if (p >= n_valid) continue;
#pragma unroll
        for (int c = 0; c < 10; ++c) {
            if ((c & 7) != g) continue;
            float v;
            if (c == 0) v = sp * y[n][0] + S.norm[6];
            else if (c < 4) v = sp * y[n][c] / S.norm[3 + c - 1];
            else  // second-order channel m = c - 4 is (k, l) = nibble m of 0x210100, 0x222110
                v = sp * y[n][c] / (S.norm[3 + ((0x210100 >> (4 * (c - 4))) & 0xf)] *
                                    S.norm[3 + ((0x222110 >> (4 * (c - 4))) & 0xf)]);
            out[10 * p + c] = v;
        }
    }
}

// ---------------------------------------------------------------- kernels --
// samples: invariants I (n x 3) -> psi, dpsi/dI (3), upper Hessian in I (6).
// The forward kernels are capped at 128 registers (4 blocks, 16 warps per
// SM): the small spill this causes costs less than the latency that 12
// warps at 168 registers could not hide (measured: 14 % faster on the batch).
__global__ void __launch_bounds__(WARPS * 32, 4) k_mlp_eval(const float *th, const float *norm, int64_t n,
                                                          const float *I, float *out)
{
    __shared__ MlpSmem S;
    __shared__ float slab[WARPS][2 * H * 8];
    load_params(S, th, norm);
    __syncthreads();
    const int w = threadIdx.x >> 5, g = (threadIdx.x & 31) >> 2;
    for (int64_t base = ((int64_t)blockIdx.x * WARPS + w) * 8; base < n; base += (int64_t)gridDim.x * WARPS * 8) {
        const int64_t s = base + g;
        float u[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) u[k] = s < n ? (I[3 * s + k] - S.norm[k]) / S.norm[3 + k] : 0.0f;
        float y[2][10];
        warp_forward8(S, u, y, slab[w]);
        store_unstandardised(S, y, base, n, out);
    }
}


// ------------------------------------------------------------- training --
constexpr int TWARPS = 2;  // warps per block of the training kernel

struct TrainWarp {            // per-warp shared memory of the training kernel
    float z1[1024], z2[1024], dz2[3][1024];      // lane-strided slabs
    __nv_bfloat16 AT[H * LDW];                   // [i][(c, s)]: dz2^T | du2_k^T
    __nv_bfloat16 BT[H * LDW];                   // [j][(c, s)]: a1^T | t1_k^T
    float gW2[H * H];                            // gradient partials of this warp
    float gW1[H * 3], gb1[H], gb2[H], gw3[H], gb3;
    float u[16][3], ty[16], tg[16][3], dY[16], dDY[16][3], y[16], dy[16][3];
    double loss;
};

// column sums over the 16 rows of a warp tile: lanes with the same t hold the
// same columns; reduce across g (lane bits 2..4)
__device__ __forceinline__ float col_sum(float v)
{
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

__global__ void __launch_bounds__(TWARPS * 32) k_mlp_grad(const float *th, const float *norm, int64_t n,
                                                          const float *I, const float *psi_t, const float *g_t,
                                                          float beta, float *part, double *part_loss)
{
    __shared__ MlpSmem S;
    extern __shared__ __align__(16) unsigned char tw_raw[];
    TrainWarp *TWs = reinterpret_cast<TrainWarp *>(tw_raw);
    load_params(S, th, norm);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    TrainWarp &W = TWs[w];
    for (int k = lane; k < H * H; k += 32) W.gW2[k] = 0.0f;
    for (int k = lane; k < H * 3; k += 32) W.gW1[k] = 0.0f;
    for (int k = lane; k < H; k += 32) W.gb1[k] = W.gb2[k] = W.gw3[k] = 0.0f;
    if (lane == 0) {
        W.gb3 = 0.0f;
        W.loss = 0.0;
    }
    __syncthreads();
    const float inv_n = 1.0f / (float)n;
    float acc[8][4];
    uint32_t a[4][4];
    float v[32];
    for (int64_t base = ((int64_t)blockIdx.x * TWARPS + w) * 16; base < n; base += (int64_t)gridDim.x * TWARPS * 16) {
        if (lane < 16) {
            const int64_t sidx = base + lane;
            const bool ok = sidx < n;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                W.u[lane][k] = ok ? (I[3 * sidx + k] - S.norm[k]) / S.norm[3 + k] : 0.0f;
                W.tg[lane][k] = ok ? g_t[3 * sidx + k] * S.norm[3 + k] / S.norm[7] : 0.0f;
            }
            W.ty[lane] = ok ? (psi_t[sidx] - S.norm[6]) / S.norm[7] : 0.0f;
        }
        __syncwarp();
        // ---- forward: z1, value and tangent channels
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            const int r = elem_row(e), j = elem_col(e);
            W.z1[e * 32 + lane] = S.b1[j] + S.W1[3 * j] * W.u[r][0] + S.W1[3 * j + 1] * W.u[r][1] + S.W1[3 * j + 2] * W.u[r][2];
        }
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                float sg, s0, s1, s2;
                silu_all(W.z1[e * 32 + lane], sg, s0, s1, s2);
                v[e] = c == 0 ? s0 : s1 * S.W1[3 * elem_col(e) + c - 1];
            }
            to_frag(v, a);
            zero(acc);
            mma_16x64(acc, a, S.W2);
            float p0 = 0.0f, p1 = 0.0f;
#pragma unroll
            for (int nn = 0; nn < 8; ++nn)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = nn * 4 + q, i = elem_col(e);
                    float wv;
                    if (c == 0) {
                        const float z2 = acc[nn][q] + S.b2[i];
                        W.z2[e * 32 + lane] = z2;
                        float sg, s0, s1, s2;
                        silu_all(z2, sg, s0, s1, s2);
                        wv = S.w3[i] * s0;
                    } else {
                        W.dz2[c - 1][e * 32 + lane] = acc[nn][q];
                        float sg, s0, s1, s2;
                        silu_all(W.z2[e * 32 + lane], sg, s0, s1, s2);
                        wv = S.w3[i] * s1 * acc[nn][q];
                    }
                    if (q < 2) p0 += wv;
                    else p1 += wv;
                }
            p0 = quad_sum(p0);
            p1 = quad_sum(p1);
            if (t == 0) {
                if (c == 0) {
                    W.y[g] = p0 + S.b3;
                    W.y[g + 8] = p1 + S.b3;
                } else {
                    W.dy[g][c - 1] = p0;
                    W.dy[g + 8][c - 1] = p1;
                }
            }
        }
        __syncwarp();
        // ---- loss and output adjoints (rows beyond n contribute nothing)
        if (lane < 16) {
            const bool ok = base + lane < n;
            const float r0 = W.y[lane] - W.ty[lane];
            float l = r0 * r0;
            W.dY[lane] = ok ? 2.0f * r0 * inv_n : 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float rk = W.dy[lane][k] - W.tg[lane][k];
                l += beta * rk * rk;
                W.dDY[lane][k] = ok ? 2.0f * beta * rk * inv_n : 0.0f;
            }
            double ls = ok ? (double)l : 0.0;
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) ls += __shfl_down_sync(0x0000ffffu, ls, o, 16);
            if (lane == 0) W.loss += ls;
        }
        __syncwarp();
        if (lane == 0) {
            float sb3 = 0.0f;
            for (int r = 0; r < 16; ++r) sb3 += W.dY[r];
            W.gb3 += sb3;
        }
        // ---- layer 2 adjoints per element: dz2, du2_k; gradients of w3, b2
        float dz2v[32], du2v[3][32];
        {
            float cw3[16], cb2[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) cw3[q] = cb2[q] = 0.0f;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int r = elem_row(e), i = elem_col(e);
                float sg, s0, s1, s2;
                silu_all(W.z2[e * 32 + lane], sg, s0, s1, s2);
                float dz = W.dY[r] * S.w3[i] * s1;
                float gw = W.dY[r] * s0;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float d = W.dz2[k][e * 32 + lane];
                    dz += W.dDY[r][k] * S.w3[i] * s2 * d;
                    du2v[k][e] = W.dDY[r][k] * S.w3[i] * s1;
                    gw += W.dDY[r][k] * s1 * d;
                }
                dz2v[e] = dz;
                // column (e >> 2, e & 1) of the lane: q index = (e >> 2) * 2 + (e & 1)
                cw3[(e >> 2) * 2 + (e & 1)] += gw;
                cb2[(e >> 2) * 2 + (e & 1)] += dz;
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float sw = col_sum(cw3[q]), sb = col_sum(cb2[q]);
                if (g == 0) {
                    const int i = 8 * (q >> 1) + 2 * t + (q & 1);
                    W.gw3[i] += sw;
                    W.gb2[i] += sb;
                }
            }
        }
        // ---- stage operands of the W2 gradient: AT[i][(c,s)], BT[j][(c,s)]
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            const int r = elem_row(e), col = elem_col(e);
            float sg, s0, s1, s2;
            silu_all(W.z1[e * 32 + lane], sg, s0, s1, s2);
            W.AT[col * LDW + r] = __float2bfloat16(dz2v[e]);
            W.BT[col * LDW + r] = __float2bfloat16(s0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                W.AT[col * LDW + 16 * (k + 1) + r] = __float2bfloat16(du2v[k][e]);
                W.BT[col * LDW + 16 * (k + 1) + r] = __float2bfloat16(s1 * S.W1[3 * col + k]);
            }
        }
        __syncwarp();
        // ---- dW2[i][j] += sum_(c,s) AT[i][(c,s)] BT[j][(c,s)]  (4 m-tiles of i)
#pragma unroll 1
        for (int mi = 0; mi < 4; ++mi) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const __nv_bfloat16 *Ar = W.AT + (mi * 16) * LDW + kk * 16;
                a[kk][0] = *reinterpret_cast<const uint32_t *>(Ar + g * LDW + 2 * t);
                a[kk][1] = *reinterpret_cast<const uint32_t *>(Ar + (g + 8) * LDW + 2 * t);
                a[kk][2] = *reinterpret_cast<const uint32_t *>(Ar + g * LDW + 2 * t + 8);
                a[kk][3] = *reinterpret_cast<const uint32_t *>(Ar + (g + 8) * LDW + 2 * t + 8);
            }
            zero(acc);
            mma_16x64(acc, a, W.BT);
#pragma unroll
            for (int nn = 0; nn < 8; ++nn)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = nn * 4 + q;
                    const int i = mi * 16 + elem_row(e), j = elem_col(e);
                    W.gW2[i * H + j] += acc[nn][q];  // each element owned by one lane
                }
        }
        // ---- layer 1 adjoints: da1 = dz2 W2, dt1_k = du2_k W2
        float dz1v[32];
        to_frag(dz2v, a);
        zero(acc);
        mma_16x64(acc, a, S.W2T);
#pragma unroll
        for (int nn = 0; nn < 8; ++nn)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = nn * 4 + q;
                float sg, s0, s1, s2;
                silu_all(W.z1[e * 32 + lane], sg, s0, s1, s2);
                dz1v[e] = acc[nn][q] * s1;
            }
        float cW1[3][16];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int q = 0; q < 16; ++q) cW1[k][q] = 0.0f;
#pragma unroll 1
        for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = du2v[k][e];
            to_frag(v, a);
            zero(acc);
            mma_16x64(acc, a, S.W2T);
#pragma unroll
            for (int nn = 0; nn < 8; ++nn)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = nn * 4 + q, j = elem_col(e);
                    float sg, s0, s1, s2;
                    silu_all(W.z1[e * 32 + lane], sg, s0, s1, s2);
                    dz1v[e] += acc[nn][q] * s2 * S.W1[3 * j + k];
                    cW1[k][nn * 2 + (q & 1)] += acc[nn][q] * s1;   // dt1_k s'(z1)
                }
        }
        float cb1[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) cb1[q] = 0.0f;
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            const int r = elem_row(e), qc = (e >> 2) * 2 + (e & 1);
            cb1[qc] += dz1v[e];
#pragma unroll
            for (int k = 0; k < 3; ++k) cW1[k][qc] += dz1v[e] * W.u[r][k];
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float sb = col_sum(cb1[q]);
            const float s0 = col_sum(cW1[0][q]), s1 = col_sum(cW1[1][q]), s2 = col_sum(cW1[2][q]);
            if (g == 0) {
                const int j = 8 * (q >> 1) + 2 * t + (q & 1);
                W.gb1[j] += sb;
                W.gW1[3 * j] += s0;
                W.gW1[3 * j + 1] += s1;
                W.gW1[3 * j + 2] += s2;
            }
        }
        __syncwarp();
    }
    __syncwarp();
    // this warp's partial gradient, in theta order
    const int wid = blockIdx.x * TWARPS + w;
    float *P = part + (int64_t)wid * NP;
    for (int k = lane; k < H * 3; k += 32) P[k] = W.gW1[k];
    for (int k = lane; k < H; k += 32) P[H * 3 + k] = W.gb1[k];
    for (int k = lane; k < H * H; k += 32) P[H * 3 + H + k] = W.gW2[k];
    for (int k = lane; k < H; k += 32) {
        P[H * 3 + H + H * H + k] = W.gb2[k];
        P[H * 3 + H + H * H + H + k] = W.gw3[k];
    }
    if (lane == 0) {
        P[NP - 1] = W.gb3;
        part_loss[wid] = W.loss / (double)n;
    }
}

// grad[p] = sum over warps of part[w][p] (fixed order); loss likewise
__global__ void k_mlp_reduce(const float *part, const double *part_loss, int n_warps, float *grad, double *loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) {
        float s = 0.0f;
        for (int w = 0; w < n_warps; ++w) s += part[(int64_t)w * NP + p];
        grad[p] = s;
    }
    if (p == 0 && loss) {
        double l = 0.0;
        for (int w = 0; w < n_warps; ++w) l += part_loss[w];
        *loss = l;
    }
}

// Adam on the FP32 master parameters
__global__ void k_mlp_adam(float *th, float *m, float *v, const float *grad, int64_t step, float lr, float b1,
                           float b2, float eps)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NP) return;
    const float gr = grad[p];
    const float mm = b1 * m[p] + (1.0f - b1) * gr;
    const float vv = b2 * v[p] + (1.0f - b2) * gr * gr;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.0f - powf(b1, (float)step)), vh = vv / (1.0f - powf(b2, (float)step));
    th[p] -= lr * mh / (sqrtf(vh) + eps);
}

// invariants of C3 = diag(F^T F, 1) and the analytic Neo-Hookean density and
// gradient in the invariants (the same density as the Neo-Hookean term)
__global__ void k_nh_targets(int64_t n, const float *F, double mu, double lam, float *I, float *psi, float *dpsi)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double f[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) f[k] = F[6 * s + k];
    const double c11 = f[0] * f[0] + f[2] * f[2] + f[4] * f[4];
    const double c22 = f[1] * f[1] + f[3] * f[3] + f[5] * f[5];
    const double c12 = f[0] * f[1] + f[2] * f[3] + f[4] * f[5];
    const double i3 = c11 * c22 - c12 * c12, i1 = c11 + c22 + 1.0, i2 = i3 + c11 + c22;
    const double lnJ = 0.5 * ::log(i3);
    I[3 * s] = (float)i1;
    I[3 * s + 1] = (float)i2;
    I[3 * s + 2] = (float)i3;
    psi[s] = (float)(0.5 * mu * (i1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ);
    dpsi[3 * s] = (float)(0.5 * mu);
    dpsi[3 * s + 1] = 0.0f;
    dpsi[3 * s + 2] = (float)((-mu + lam * lnJ) / (2.0 * i3));
}

// per-triangle network table in unit order (the tiles' order and vertex
// rotation): psi, dpsi/dI, upper Hessian in I
__global__ void __launch_bounds__(WARPS * 32, 4) k_mlp_tri(const float *th, const float *norm, int64_t nT,
                                                         const int32_t *verts, const float *rest, const float *x,
                                                         float *table)
{
    __shared__ MlpSmem S;
    __shared__ float slab[WARPS][2 * H * 8];
    load_params(S, th, norm);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2;
    const int64_t stride = (int64_t)gridDim.x * WARPS * 8;
    // lanes 0..7 load the positions and rest data of triangle base + lane;
    // the next iteration's are loaded while the network runs
    auto load = [&](int64_t bb, float (&xv)[9], float (&D)[4]) {
        const int64_t p = bb + (lane & 7);
        if (lane < 8 && p < nT) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t v = verts[3 * p + c];
#pragma unroll
                for (int d = 0; d < 3; ++d) xv[3 * c + d] = x[3 * v + d];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) D[k] = rest[k * nT + p];
        } else {
#pragma unroll
            for (int k = 0; k < 9; ++k) xv[k] = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) D[k] = 0.0f;
        }
    };
    float xv[9], D[4];
    load(((int64_t)blockIdx.x * WARPS + w) * 8, xv, D);
    for (int64_t base = ((int64_t)blockIdx.x * WARPS + w) * 8; base < nT; base += stride) {
        // lanes 0..7 form the invariants of triangles base + lane
        float uu[3] = {0.0f, 0.0f, 0.0f};
        if (lane < 8 && base + lane < nT) {
            float c11 = 0.0f, c22 = 0.0f, c12 = 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float u1 = xv[3 + d] - xv[d], w1 = xv[6 + d] - xv[d];
                const float f1 = u1 * D[0] + w1 * D[2], f2 = u1 * D[1] + w1 * D[3];
                c11 += f1 * f1;
                c22 += f2 * f2;
                c12 += f1 * f2;
            }
            const float i3 = c11 * c22 - c12 * c12;
            const float I3[3] = {c11 + c22 + 1.0f, i3 + c11 + c22, i3};
#pragma unroll
            for (int k = 0; k < 3; ++k) uu[k] = (I3[k] - S.norm[k]) / S.norm[3 + k];
        }
        load(base + stride, xv, D);
        float u[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) u[k] = __shfl_sync(0xffffffffu, uu[k], g);
        float y[2][10];
        warp_forward8(S, u, y, slab[w]);
        store_unstandardised(S, y, base, nT, table);
    }
}

// ---------------------------------------------- tcgen05 network variant --
// The per-triangle network of k_mlp_tri on the fifth-generation tensor
// cores: the contractions are tcgen05.mma (kind::f16, BF16 operands from
// shared memory, FP32 accumulators in tensor memory), issued by one thread
// and completed on an mbarrier; the elementwise work stays on the FP32 pipes.
// A tile is 128 triangles (the MMA's M), one TMEM lane per triangle:
//   1. layer 1 in FP32, its value and 3 tangents written as four BF16 A
//      operands (128 x 64 each) in the K-major canonical layout;
//   2. z2 of the 4 channels, D_c = A_c W2^T, into TMEM columns 64 c .. 64 c + 63
//      (16 MMAs of 128 x 64 x 16);
//   3. from TMEM: silu of z2 and its derivatives, the value, gradient and
//      first second-order part, and rho = w3 silu'(z2) written as a BF16 A
//      operand over channel 0's;
//   4. r = rho W2 (4 MMAs) into columns 0 .. 63, then the second part
//      sum_n r_n silu''(z1_n) W1_nk W1_nl.
// Two threads per triangle: warps w and w + 4 read the same TMEM lanes
// (a warp reaches lanes 32 (w mod 4) ..); the first takes units 0-31, the
// second 32-63, and their partial outputs meet in shared memory.
// Canonical K-major layout without swizzle: element (row, k) at byte
// (row / 8) 128 + (k / 8) LBO + (row % 8) 16 + (k % 8) 2, i.e. 8 x 16-byte
// core matrices, row groups 128 bytes apart (the descriptor's SBO), K chunks
// LBO apart.
namespace tc {
constexpr int TILE = 128, THREADS = 256, HALF = H / 2;
constexpr uint32_t A_LBO = (TILE / 8) * 128, B_LBO = (H / 8) * 128;
constexpr uint32_t A_BYTES = TILE * H * 2, B_BYTES = H * H * 2;
constexpr uint32_t SMEM = 4 * A_BYTES + 2 * B_BYTES;  // 80 KB: two blocks per SM, 256 TMEM columns each
constexpr uint32_t TMEM_COLS = 256;
// instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, N, M
constexpr uint32_t IDESC = umma_idesc_bf16(TILE, H);

__device__ __forceinline__ uint32_t canon(int row, int k, uint32_t lbo) { return umma_canon(row, k, lbo); }
// shared-memory matrix descriptor: start, LBO, SBO = 128 (bytes >> 4), the
// descriptor version bit, no swizzle
__device__ __forceinline__ uint64_t sdesc(const void *p, uint32_t lbo)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    return (uint64_t)((a >> 4) & 0x3FFFu) | (uint64_t)((lbo >> 4) & 0x3FFFu) << 16 | (uint64_t)(128u >> 4) << 32 |
           (uint64_t)1 << 46;
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, bool acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                 "l"(a), "l"(b), "r"(IDESC), "r"((uint32_t)acc)
                 : "memory");
}
__device__ __forceinline__ void commit(uint64_t *bar)
{
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b) : "memory");
}
// wait for the given phase parity; gives up after about a second
__device__ __forceinline__ bool wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    for (int it = 0; it < (1 << 20); ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(b), "r"(parity), "r"(1000u)
                     : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 8 consecutive FP32 columns of this thread's TMEM lane; the load and its
// wait in one statement, so that no use of the registers precedes the wait
__device__ __forceinline__ void ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}
// 8 columns at each of 4 column offsets (the four channels), one wait
__device__ __forceinline__ void ld8x4(uint32_t t0, uint32_t t1, uint32_t t2, uint32_t t3, float (&v)[4][8])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%33];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%34];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%35];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3)
        : "memory");
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int q = 0; q < 8; ++q) v[c][q] = __uint_as_float(r[8 * c + q]);
}
// the logistic function with the fast divide intrinsic (about 2 ulp; the
// activations are rounded to BF16 before every contraction), and the SiLU
// formulas of silu_all on it: value and first derivative (layer 1), all
// three (layer 2), the second derivative from a kept sigma (reverse part)
__device__ __forceinline__ float sigm(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
__device__ __forceinline__ void silu01(float z, float sg, float &s, float &s1)
{
    s = z * sg;
    s1 = sg * (1.0f + z * (1.0f - sg));
}
__device__ __forceinline__ float silu2(float z, float sg) { return sg * (1.0f - sg) * (2.0f + z * (1.0f - 2.0f * sg)); }
// 8 BF16 values into one 16-byte row piece of a canonical operand
__device__ __forceinline__ void st8(unsigned char *dst, const float (&v)[8])
{
    uint4 w;
    w.x = pack_bf16(v[0], v[1]);
    w.y = pack_bf16(v[2], v[3]);
    w.z = pack_bf16(v[4], v[5]);
    w.w = pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4 *>(dst) = w;
}
}  // namespace tc

__global__ void __launch_bounds__(tc::THREADS, 2) k_mlp_tri_tc(const float *th, const float *norm, int64_t nT,
                                                                const int32_t *verts, const float *rest,
                                                                const float *x, float *table, int *status)
{
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    __shared__ float W1s[H * 3], b1s[H], b2s[H], w3s[H], b3s, norms[8];
    __shared__ float part[TILE][10];  // the second half's partial outputs
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t taddr_s;
    unsigned char *Ac = smem_tc;                      // 4 operands: a1, da1/du_0..2 (rho over a1's)
    unsigned char *Bz = smem_tc + 4 * A_BYTES;        // W2 (rows: layer-2 units, K: layer-1 units)
    unsigned char *Br = Bz + B_BYTES;                 // W2^T (rows: layer-1 units, K: layer-2 units)
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int row = 32 * (w & 3) + lane;  // this thread's triangle within the tile, its TMEM lane
    const int u0 = (w >> 2) * HALF;       // first unit of this thread's half
    // parameters, BF16-rounded as the other kernels use them
    {
        const float *W1 = th, *b1 = W1 + H * 3, *W2 = b1 + H, *b2 = W2 + H * H, *w3 = b2 + H, *b3 = w3 + H;
        for (int k = tid; k < H * H; k += THREADS) {
            const int i = k / H, j = k % H;
            const __nv_bfloat16 v = __float2bfloat16(W2[k]);
            *reinterpret_cast<__nv_bfloat16 *>(Bz + canon(i, j, B_LBO)) = v;
            *reinterpret_cast<__nv_bfloat16 *>(Br + canon(j, i, B_LBO)) = v;
        }
        for (int k = tid; k < H * 3; k += THREADS) W1s[k] = bf16r(W1[k]);
        for (int k = tid; k < H; k += THREADS) {
            b1s[k] = bf16r(b1[k]);
            b2s[k] = bf16r(b2[k]);
            w3s[k] = bf16r(w3[k]);
        }
        if (tid == 0) b3s = bf16r(b3[0]);
        if (tid < 8) norms[tid] = norm[tid];
    }
    if (w == 0) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&taddr_s);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = taddr_s, tlane = tbase + ((uint32_t)(32 * (w & 3)) << 16);
    constexpr int K2[6] = {0, 0, 1, 0, 1, 2}, L2[6] = {0, 1, 1, 2, 2, 2};
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t t0 = (int64_t)blockIdx.x * TILE; t0 < nT && ok; t0 += (int64_t)gridDim.x * TILE) {
        const int64_t p = t0 + row;
        // invariants of triangle p, standardised (zero past the end)
        float u[3] = {0.0f, 0.0f, 0.0f};
        if (p < nT) {
            float xv[9], D[4];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t v = verts[3 * p + c];
#pragma unroll
                for (int d = 0; d < 3; ++d) xv[3 * c + d] = x[3 * v + d];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) D[k] = rest[k * nT + p];
            float c11 = 0.0f, c22 = 0.0f, c12 = 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float e1 = xv[3 + d] - xv[d], e2 = xv[6 + d] - xv[d];
                const float f1 = e1 * D[0] + e2 * D[2], f2 = e1 * D[1] + e2 * D[3];
                c11 += f1 * f1;
                c22 += f2 * f2;
                c12 += f1 * f2;
            }
            const float i3 = c11 * c22 - c12 * c12;
            const float I3[3] = {c11 + c22 + 1.0f, i3 + c11 + c22, i3};
#pragma unroll
            for (int k = 0; k < 3; ++k) u[k] = (I3[k] - norms[k]) / norms[3 + k];
        }
        // 1. layer 1 of this half's units: value and tangents as BF16
        // operands; sigma(z1) kept in registers for the reverse part
        float sg1[HALF];
#pragma unroll
        for (int kb = 0; kb < HALF / 8; ++kb) {
            float v[4][8];
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int i = u0 + 8 * kb + o;
                const float wa = W1s[3 * i], wb = W1s[3 * i + 1], wc = W1s[3 * i + 2];
                const float z1 = b1s[i] + wa * u[0] + wb * u[1] + wc * u[2];
                sg1[8 * kb + o] = sigm(z1);
                float s0, s1;
                silu01(z1, sg1[8 * kb + o], s0, s1);
                v[0][o] = s0;
                v[1][o] = s1 * wa;
                v[2][o] = s1 * wb;
                v[3][o] = s1 * wc;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) st8(Ac + c * A_BYTES + canon(row, u0 + 8 * kb, A_LBO), v[c]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
        // 2. z2 of the four channels
        if (tid == 0) {
            fence_after();
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int j = 0; j < H / 16; ++j)
                    mma(tbase + 64 * c, sdesc(Ac + c * A_BYTES + 2 * j * A_LBO, A_LBO), sdesc(Bz + 2 * j * B_LBO, B_LBO),
                        j > 0);
            commit(&bar);
        }
        ok = __syncthreads_and(wait(&bar, phase & 1u));
        if (!ok) wait(&bar, phase & 1u);  // bounded again: the MMAs in flight land before the TMEM is freed
        ++phase;
        fence_after();
        if (!ok) break;
        // 3. layer 2 and the output layer for this half's units; rho as an operand
        float y[10];
#pragma unroll
        for (int c = 0; c < 10; ++c) y[c] = 0.0f;
#pragma unroll 1
        for (int kb = 0; kb < HALF / 8; ++kb) {
            const int j0 = u0 + 8 * kb;
            float z[4][8];
            ld8x4(tlane + (uint32_t)j0, tlane + (uint32_t)(64 + j0), tlane + (uint32_t)(128 + j0),
                  tlane + (uint32_t)(192 + j0), z);
            float rho[8];
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int j = j0 + o;
                const float z2 = z[0][o] + b2s[j], sg = sigm(z2);
                float s0, s1;
                silu01(z2, sg, s0, s1);
                const float s2 = silu2(z2, sg);
                const float wj = w3s[j], d[3] = {z[1][o], z[2][o], z[3][o]};
                const float g1 = wj * s1, g2 = wj * s2;
                const float e[3] = {g2 * d[0], g2 * d[1], g2 * d[2]};
                y[0] += wj * s0;
#pragma unroll
                for (int k = 0; k < 3; ++k) y[1 + k] += g1 * d[k];
#pragma unroll
                for (int m = 0; m < 6; ++m) y[4 + m] += e[K2[m]] * d[L2[m]];
                rho[o] = g1;
            }
            st8(Ac + canon(row, j0, A_LBO), rho);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
        // 4. r = rho W2 (row = triangle, column = layer-1 unit n)
        if (tid == 0) {
            fence_after();
#pragma unroll
            for (int j = 0; j < H / 16; ++j)
                mma(tbase, sdesc(Ac + 2 * j * A_LBO, A_LBO), sdesc(Br + 2 * j * B_LBO, B_LBO), j > 0);
            commit(&bar);
        }
        ok = __syncthreads_and(wait(&bar, phase & 1u));
        if (!ok) wait(&bar, phase & 1u);  // as above
        ++phase;
        fence_after();
        if (!ok) break;
#pragma unroll
        for (int kb = 0; kb < HALF / 8; ++kb) {
            const int n0 = u0 + 8 * kb;
            float r[8];
            ld8(tlane + (uint32_t)n0, r);
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int n = n0 + o;
                const float wa = W1s[3 * n], wb = W1s[3 * n + 1], wc = W1s[3 * n + 2];
                const float q = r[o] * silu2(b1s[n] + wa * u[0] + wb * u[1] + wc * u[2], sg1[8 * kb + o]);
                const float wk[3] = {wa, wb, wc}, qk[3] = {q * wa, q * wb, q * wc};
#pragma unroll
                for (int m = 0; m < 6; ++m) y[4 + m] += qk[K2[m]] * wk[L2[m]];
            }
        }
        // the two halves of each triangle meet; the first half stores
        if (w >= 4)
#pragma unroll
            for (int c = 0; c < 10; ++c) part[row][c] = y[c];
        fence_before();
        __syncthreads();
        if (w < 4 && p < nT) {
            const float sp = norms[7];
#pragma unroll
            for (int c = 0; c < 10; ++c) {
                const float v = y[c] + part[row][c] + (c == 0 ? b3s : 0.0f);
                float o;
                if (c == 0) o = sp * v + norms[6];
                else if (c < 4) o = sp * v / norms[3 + c - 1];
                else o = sp * v / (norms[3 + K2[c - 4]] * norms[3 + L2[c - 4]]);
                table[10 * p + c] = o;
            }
        }
    }
    if (!ok && tid == 0) atomicOr(status, ST_TIMEOUT);
    fence_before();
    __syncthreads();
    if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
}

}  // namespace

// launchers used by api.cpp
adm_status mlp_eval_samples(const float *th, const float *norm, int64_t n, const float *I, float *out,
                            cudaStream_t s)
{
    const int64_t blocks = std::min<int64_t>((n + WARPS * 8 - 1) / (WARPS * 8), 152 * 8);
    if (blocks > 0) k_mlp_eval<<<(unsigned)blocks, WARPS * 32, 0, s>>>(th, norm, n, I, out);
    return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}


size_t mlp_workspace_bytes()
{
    return (size_t)152 * TWARPS * (NP * sizeof(float) + sizeof(double)) + 256;
}

adm_status mlp_loss_grad(const float *th, const float *norm, int64_t n, const float *I, const float *psi,
                         const float *g, float beta, double *loss, float *grad, void *ws, size_t ws_bytes,
                         cudaStream_t s)
{
    if (n <= 0 || ws_bytes < mlp_workspace_bytes()) return ADM_ERR_ARG;
    const int blocks = 152;
    float *part = (float *)ws;
    double *part_loss = (double *)((char *)ws + (((size_t)blocks * TWARPS * NP * sizeof(float) + 255) & ~(size_t)255));
    const size_t dyn = TWARPS * sizeof(TrainWarp);
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    k_mlp_grad<<<blocks, TWARPS * 32, dyn, s>>>(th, norm, n, I, psi, g, beta, part, part_loss);
    k_mlp_reduce<<<(NP + 255) / 256, 256, 0, s>>>(part, part_loss, blocks * TWARPS, grad, loss);
    return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}

adm_status mlp_adam(float *th, float *m, float *v, const float *grad, int64_t step, float lr, float b1, float b2,
                    float eps, cudaStream_t s)
{
    k_mlp_adam<<<(NP + 255) / 256, 256, 0, s>>>(th, m, v, grad, step, lr, b1, b2, eps);
    return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}

adm_status mlp_nh_targets(int64_t n, const float *F, double mu, double lam, float *I, float *psi, float *dpsi,
                          cudaStream_t s)
{
    if (n > 0) k_nh_targets<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, F, mu, lam, I, psi, dpsi);
    return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}

adm_status mlp_triangle_table(const float *th, const float *norm, int64_t nT, const int32_t *verts,
                              const float *rest_tiled, const float *x, float *table, int tc_net, int *status,
                              cudaStream_t s)
{
    if (tc_net) {
        // persistent: two blocks per SM (shared memory allows no third, so
        // the 256 TMEM columns of each always fit)
        int dev = 0, n_sm = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        const int64_t blocks = std::min<int64_t>((nT + tc::TILE - 1) / tc::TILE, 2 * (int64_t)n_sm);
        cudaFuncSetAttribute(k_mlp_tri_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM);
        if (blocks > 0)
            k_mlp_tri_tc<<<(unsigned)blocks, tc::THREADS, tc::SMEM, s>>>(th, norm, nT, verts, rest_tiled, x, table,
                                                                         status);
        return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
    }
    const int64_t blocks = std::min<int64_t>((nT + WARPS * 8 - 1) / (WARPS * 8), 152 * 8);
    if (blocks > 0) k_mlp_tri<<<(unsigned)blocks, WARPS * 32, 0, s>>>(th, norm, nT, verts, rest_tiled, x, table);
    return cudaGetLastError() == cudaSuccess ? ADM_OK : ADM_ERR_CUDA;
}

}  // namespace adm

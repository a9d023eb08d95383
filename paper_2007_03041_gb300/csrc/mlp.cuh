// WENO-weight network of the learned weight path (the paper has no learned
// component): 5 stencil values -> 32 -> 32 -> 3, tanh-form GELU after both
// hidden layers, softmax output = the nonlinear weights w_r of the WENO
// combination J = sum_r w_r J^{(r)} (Sec. 2.4).
//
// Tensor cores: every layer is a warp-level BF16 matrix product with FP32
// accumulation (mma.sync m16n8k16) over 16 stencils at a time.  A layer's
// accumulator fragments are re-packed in registers as the A operand of the
// next one (the two layouts coincide), the biases enter as the accumulators'
// initial values, and the weight fragments stay in registers across groups.
//
// Fragment layouts of m16n8k16 (g = lane/4, t = lane%4):
//   A (16x16, row): a0a1 = A[g][2t..2t+1], a2a3 = A[g+8][2t..], a4a5 = A[g][2t+8..],
//                   a6a7 = A[g+8][2t+8..]
//   B (16x8, col):  b0b1 = B[2t..2t+1][g], b2b3 = B[2t+8..2t+9][g]
//   C (16x8):       c0c1 = C[g][2t..2t+1], c2c3 = C[g+8][2t..2t+1]
//
// Conventions shared with the training kernels: network inputs are the
// stencil values minus the middle one, divided by their largest magnitude
// (+1e-30); inputs and hidden activations are rounded to BF16 before each
// product; GELU(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace molt {

// FP32 master parameters: W1 (32x5), b1 (32), W2 (32x32), b2 (32), W3 (3x32), b3 (3).
constexpr int kMlpParams = 1347;
constexpr int kOffW1 = 0, kOffB1 = 160, kOffW2 = 192, kOffB2 = 1216, kOffW3 = 1248, kOffB3 = 1344;

// BF16 weights in the layout the library takes (row-major, zero padded).
struct MlpBlob {
  __nv_bfloat16 W1[32][16];   // inputs 0..4 used
  __nv_bfloat16 W2[32][32];
  __nv_bfloat16 W3[8][32];    // outputs 0..2 used
  __nv_bfloat16 b1[32], b2[32], b3[8];
};
static_assert(sizeof(MlpBlob) == 3728, "blob layout");

// Shared-memory copy with padded rows: the B-fragment loads of a warp (word
// 12g+t resp. 20g+t) fall in 32 distinct banks.
constexpr int kLd1 = 24, kLd2 = 40;
struct MlpNet {
  __nv_bfloat16 W1[32][kLd1];
  __nv_bfloat16 W2[32][kLd2];
  __nv_bfloat16 W3[8][kLd2];
  float b1[32], b2[32], b3[8];
};

__device__ __forceinline__ void mlp_load_net(MlpNet& s, const MlpBlob* g) {
  const __nv_bfloat16 z = __float2bfloat16(0.f);
  for (int i = threadIdx.x; i < 32 * kLd1; i += blockDim.x) {
    const int r = i / kLd1, c = i - r * kLd1;
    s.W1[r][c] = c < 16 ? g->W1[r][c] : z;
  }
  for (int i = threadIdx.x; i < 32 * kLd2; i += blockDim.x) {
    const int r = i / kLd2, c = i - r * kLd2;
    s.W2[r][c] = c < 32 ? g->W2[r][c] : z;
  }
  for (int i = threadIdx.x; i < 8 * kLd2; i += blockDim.x) {
    const int r = i / kLd2, c = i - r * kLd2;
    s.W3[r][c] = c < 32 ? g->W3[r][c] : z;
  }
  for (int i = threadIdx.x; i < 32; i += blockDim.x) {
    s.b1[i] = __bfloat162float(g->b1[i]);
    s.b2[i] = __bfloat162float(g->b2[i]);
    if (i < 8) s.b3[i] = __bfloat162float(g->b3[i]);
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float kGeluC = 0.7978845608028654f;   // sqrt(2/pi)
constexpr float kGeluA = 0.044715f;

__device__ __forceinline__ float gelu(float z) {
  return 0.5f * z * (1.f + tanh_approx(kGeluC * fmaf(kGeluA * z, z * z, z)));
}

__device__ __forceinline__ float gelu_grad(float z) {
  const float th = tanh_approx(kGeluC * fmaf(kGeluA * z, z * z, z));
  return 0.5f * (1.f + th) + 0.5f * z * (1.f - th * th) * kGeluC * fmaf(3.f * kGeluA, z * z, 1.f);
}

// Weight fragments and biases of one lane, held in registers across groups.
struct MlpRegs {
  uint32_t w1[4];          // W1 rows nt*8+g, cols 2t..2t+1 (cols 8..15 are zero)
  uint32_t w2[4][2][2];    // W2 rows nt*8+g, k-tile kk
  uint32_t w3[2][2];       // W3 row g, k-tile kk
  float b1[4][2], b2[4][2], b3[2];
};

__device__ __forceinline__ void mlp_load_regs(const MlpNet& s, int lane, MlpRegs& R) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    R.w1[nt] = ld32(&s.W1[nt * 8 + g][2 * t]);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      R.w2[nt][kk][0] = ld32(&s.W2[nt * 8 + g][16 * kk + 2 * t]);
      R.w2[nt][kk][1] = ld32(&s.W2[nt * 8 + g][16 * kk + 8 + 2 * t]);
    }
    R.b1[nt][0] = s.b1[nt * 8 + 2 * t];
    R.b1[nt][1] = s.b1[nt * 8 + 2 * t + 1];
    R.b2[nt][0] = s.b2[nt * 8 + 2 * t];
    R.b2[nt][1] = s.b2[nt * 8 + 2 * t + 1];
  }
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    R.w3[kk][0] = ld32(&s.W3[g][16 * kk + 2 * t]);
    R.w3[kk][1] = ld32(&s.W3[g][16 * kk + 8 + 2 * t]);
  }
  R.b3[0] = s.b3[2 * t];
  R.b3[1] = s.b3[2 * t + 1];
}

// Network inputs of a 5-value stencil.
__device__ __forceinline__ void mlp_normalise(const float (&v)[5], float (&x)[5]) {
  float m = 0.f;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    x[j] = v[j] - v[2];
    m = fmaxf(m, fabsf(x[j]));
  }
  const float inv = 1.f / (m + 1e-30f);
#pragma unroll
  for (int j = 0; j < 5; ++j) x[j] *= inv;
}

// A fragment of the inputs of stencils g (x0) and g+8 (x1): columns 0..4 of 16.
__device__ __forceinline__ void mlp_input_frag(const float (&x0)[5], const float (&x1)[5], int t, uint32_t (&a)[4]) {
  const float l0 = t == 0 ? x0[0] : (t == 1 ? x0[2] : (t == 2 ? x0[4] : 0.f));
  const float h0 = t == 0 ? x0[1] : (t == 1 ? x0[3] : 0.f);
  const float l1 = t == 0 ? x1[0] : (t == 1 ? x1[2] : (t == 2 ? x1[4] : 0.f));
  const float h1 = t == 0 ? x1[1] : (t == 1 ? x1[3] : 0.f);
  a[0] = pack_bf16(l0, h0);
  a[1] = pack_bf16(l1, h1);
  a[2] = 0u;
  a[3] = 0u;
}

// Intermediates of one forward pass (the backward pass reads them).
struct MlpCache {
  float z1[4][4], z2[4][4];     // pre-activations, C layout per n-tile
  uint32_t a1[2][4], a2[2][4];  // BF16 activations, A layout per k-tile
};

// GELU of a pair of pre-activations in packed FP32x2 arithmetic (the same
// formula as gelu(), with 0.5z(1+t) taken as the FMA 0.5z + 0.5z*t), packed
// as BF16x2.
__device__ __forceinline__ uint32_t gelu2_pack(float z0, float z1) {
  const float2 z = make_float2(z0, z1);
  const float2 zz = __fmul2_rn(z, z);
  const float2 az = __fmul2_rn(make_float2(kGeluA, kGeluA), z);
  const float2 v = __fmul2_rn(make_float2(kGeluC, kGeluC), __ffma2_rn(az, zz, z));
  const float2 t = make_float2(tanh_approx(v.x), tanh_approx(v.y));
  const float2 hz = __fmul2_rn(make_float2(0.5f, 0.5f), z);
  const float2 g = __ffma2_rn(hz, t, hz);
  return pack_bf16(g.x, g.y);
}

__device__ __forceinline__ void gelu_pack(const float (&z)[4][4], uint32_t (&a)[2][4]) {
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    a[kk][0] = gelu2_pack(z[2 * kk][0], z[2 * kk][1]);
    a[kk][1] = gelu2_pack(z[2 * kk][2], z[2 * kk][3]);
    a[kk][2] = gelu2_pack(z[2 * kk + 1][0], z[2 * kk + 1][1]);
    a[kk][3] = gelu2_pack(z[2 * kk + 1][2], z[2 * kk + 1][3]);
  }
}

__device__ __forceinline__ void softmax3(float l0, float l1, float l2, float (&p)[3]) {
  const float m = fmaxf(l0, fmaxf(l1, l2));
  const float e0 = __expf(l0 - m), e1 = __expf(l1 - m), e2 = __expf(l2 - m);
  const float inv = 1.f / (e0 + e1 + e2);
  p[0] = e0 * inv;
  p[1] = e1 * inv;
  p[2] = e2 * inv;
}

// Forward pass of 16 stencils: rows g and g+8 of the warp's group.  On return
// every lane of row group g holds the outputs p0 (row g) and p1 (row g+8).
__device__ __forceinline__ void mlp_forward16(const MlpRegs& R, const uint32_t (&xa)[4], MlpCache& f,
                                              float (&p0)[3], float (&p1)[3]) {
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    float c[4] = {R.b1[nt][0], R.b1[nt][1], R.b1[nt][0], R.b1[nt][1]};
    mma16816(c, xa, R.w1[nt], 0u);
#pragma unroll
    for (int i = 0; i < 4; ++i) f.z1[nt][i] = c[i];
  }
  gelu_pack(f.z1, f.a1);
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    float c[4] = {R.b2[nt][0], R.b2[nt][1], R.b2[nt][0], R.b2[nt][1]};
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) mma16816(c, f.a1[kk], R.w2[nt][kk][0], R.w2[nt][kk][1]);
#pragma unroll
    for (int i = 0; i < 4; ++i) f.z2[nt][i] = c[i];
  }
  gelu_pack(f.z2, f.a2);
  float c[4] = {R.b3[0], R.b3[1], R.b3[0], R.b3[1]};
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) mma16816(c, f.a2[kk], R.w3[kk][0], R.w3[kk][1]);
  // logits 0 and 1 sit in lane t = 0 of the row group, logit 2 in lane t = 1
  const int base = (threadIdx.x & 31) & ~3;
  const float l00 = __shfl_sync(0xffffffffu, c[0], base), l01 = __shfl_sync(0xffffffffu, c[1], base);
  const float l02 = __shfl_sync(0xffffffffu, c[0], base + 1);
  const float l10 = __shfl_sync(0xffffffffu, c[2], base), l11 = __shfl_sync(0xffffffffu, c[3], base);
  const float l12 = __shfl_sync(0xffffffffu, c[2], base + 1);
  softmax3(l00, l01, l02, p0);
  softmax3(l10, l11, l12, p1);
}

// WENO-Z weights of a 5-value stencil w[0..4] (J_R orientation, offsets
// -3..1; Sec. 2.4): beta_r of the quadratic through substencil r,
// w~_r = d_r (1 + tau/(eps + beta_r)), tau = |beta_0 - beta_2|, normalised.
// Same closed forms for beta_r as the WENO-Z sweeps.
__device__ __forceinline__ void wenoz_omega(const float (&w)[5], const float (&d)[3], float (&om)[3]) {
  float beta[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float a = w[r], b = w[r + 1], c = w[r + 2];
    const float s1 = 0.5f * (c - a);
    const float s2 = a - 2.f * b + c;
    const float k = r == 0 ? 3.f : (r == 1 ? 1.f : -1.f);
    const float m = r == 0 ? float(10.0 / 3.0) : float(4.0 / 3.0);
    beta[r] = s1 * s1 + k * s1 * s2 + m * s2 * s2;
  }
  const float tau = fabsf(beta[0] - beta[2]);
  float sum = 0.f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float rc;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rc) : "f"(1e-6f + beta[r]));
    om[r] = fmaf(d[r] * tau, rc, d[r]);      // d_r (1 + tau/(eps+beta_r))
    sum += om[r];
  }
  float inv;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(sum));
#pragma unroll
  for (int r = 0; r < 3; ++r) om[r] *= inv;
}

constexpr float kFallbackTol = 1e-2f;

// Final weights of one stencil: the network's, or WENO-Z's where the two
// differ by more than kFallbackTol in any component.  Returns true on fallback.
__device__ __forceinline__ bool mlp_final_weights(const float (&v)[5], const float (&p)[3], const float (&d)[3],
                                                  float (&w)[3]) {
  float om[3];
  wenoz_omega(v, d, om);
  const float res = fmaxf(fabsf(p[0] - om[0]), fmaxf(fabsf(p[1] - om[1]), fabsf(p[2] - om[2])));
  const bool fb = !(res <= kFallbackTol);   // a non-finite output falls back too
#pragma unroll
  for (int r = 0; r < 3; ++r) w[r] = fb ? om[r] : p[r];
  return fb;
}

}  // namespace molt

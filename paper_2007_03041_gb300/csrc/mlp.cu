// Training and evaluation kernels of the WENO-weight network (learned weight
// path; the paper has no learned component) and their C-ABI entry points.
//
//   mlp_forward_kernel  network weights of raw stencils (optionally with the
//                       WENO-Z fallback), one warp per 16 stencils;
//   mlp_grad_kernel     forward + backward pass and the mean-squared loss:
//                       every product of the backward pass is a BF16 tensor-
//                       core product with FP32 accumulation; the weight
//                       gradients contract over the 16 stencils of a group,
//                       with the transposed operands staged per warp in
//                       shared memory; per-warp register accumulators are
//                       reduced per CTA in shared memory, then added to the
//                       global gradient;
//   mlp_adam_kernel     Adam step on the FP32 master parameters + BF16 blob;
//   mlp_pack_kernel     FP32 master parameters -> BF16 blob;
//   mlp_harvest_kernel  training stencils (and WENO-Z targets) gathered from
//                       a periodic 2-D state.
#include <cuda_runtime.h>

#include <cmath>

#include "coeffs.h"
#include "molt.h"
#include "mlp.cuh"

using namespace molt;

namespace {

constexpr int kGradWarps = 4;   // warps per CTA of the gradient kernel

int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// FP32 master parameters -> BF16 blob, by all threads of one CTA.  The blob
// is one array of BF16: W1 (32x16), W2 (32x32), W3 (8x32), b1, b2, b3 (8).
__device__ void pack_blob(const float* theta, MlpBlob* blob) {
  __nv_bfloat16* o = &blob->W1[0][0];
  for (int f = threadIdx.x; f < int(sizeof(MlpBlob) / 2); f += blockDim.x) {
    float v = 0.f;
    if (f < 512) {
      const int r = f >> 4, c = f & 15;
      if (c < 5) v = theta[kOffW1 + r * 5 + c];
    } else if (f < 1536) {
      v = theta[kOffW2 + (f - 512)];
    } else if (f < 1792) {
      const int r = (f - 1536) >> 5, c = (f - 1536) & 31;
      if (r < 3) v = theta[kOffW3 + r * 32 + c];
    } else if (f < 1824) {
      v = theta[kOffB1 + (f - 1792)];
    } else if (f < 1856) {
      v = theta[kOffB2 + (f - 1824)];
    } else if (f - 1856 < 3) {
      v = theta[kOffB3 + (f - 1856)];
    }
    o[f] = __float2bfloat16_rn(v);
  }
}

__global__ void mlp_pack_kernel(const float* __restrict__ theta, MlpBlob* blob) { pack_blob(theta, blob); }

// b1, b2 and their complements 1-b1, 1-b2 come rounded from FP64 (1 - 0.999f
// in FP32 would be off by 1.3e-5 relative).
__global__ void mlp_adam_kernel(float* theta, float* m, float* v, const float* __restrict__ grad, float lr, float b1,
                                float omb1, float b2, float omb2, float eps, float bc1, float bc2, MlpBlob* blob) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    const float g = grad[i];
    const float mi = fmaf(b1, m[i], omb1 * g);
    const float vi = fmaf(b2, v[i], omb2 * g * g);
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
  __syncthreads();
  pack_blob(theta, blob);
}

__device__ __forceinline__ void load_stencil(const float* x, long long row, float (&v)[5]) {
#pragma unroll
  for (int j = 0; j < 5; ++j) v[j] = x[row * 5 + j];
}

__global__ void __launch_bounds__(256) mlp_forward_kernel(const MlpBlob* blob, const float* __restrict__ x,
                                                          long long n, float d0, float d1, float d2, int fallback,
                                                          float* __restrict__ w, unsigned long long* nfb) {
  __shared__ MlpNet net;
  mlp_load_net(net, blob);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  MlpRegs R;
  mlp_load_regs(net, lane, R);
  const float d[3] = {d0, d1, d2};
  unsigned fb = 0;
  const long long groups = (n + 15) / 16;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long grp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; grp < groups; grp += nw) {
    const long long r0 = grp * 16 + g, r1 = r0 + 8;
    float v0[5], v1[5];
    load_stencil(x, r0 < n ? r0 : n - 1, v0);
    load_stencil(x, r1 < n ? r1 : n - 1, v1);
    float x0[5], x1[5];
    mlp_normalise(v0, x0);
    mlp_normalise(v1, x1);
    uint32_t xa[4];
    mlp_input_frag(x0, x1, t, xa);
    MlpCache f;
    float p0[3], p1[3];
    mlp_forward16(R, xa, f, p0, p1);
    const long long r = t == 0 ? r0 : r1;
    if (t < 2 && r < n) {
      float v[5], p[3], ww[3];
#pragma unroll
      for (int j = 0; j < 5; ++j) v[j] = t == 0 ? v0[j] : v1[j];
#pragma unroll
      for (int k = 0; k < 3; ++k) p[k] = t == 0 ? p0[k] : p1[k];
      if (fallback) {
        fb += mlp_final_weights(v, p, d, ww) ? 1u : 0u;
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) ww[k] = p[k];
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) w[r * 3 + k] = ww[k];
    }
  }
  if (fallback && nfb) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fb += __shfl_xor_sync(0xffffffffu, fb, o);
    if (lane == 0 && fb) atomicAdd(nfb, (unsigned long long)fb);
  }
}

// Per-warp staging of the operands the weight gradients read transposed.
struct WarpStage {
  __nv_bfloat16 X[16][8];       // BF16 inputs (rows x in; 5..7 zero)
  __nv_bfloat16 A1[16][kLd2];   // hidden activations (rows x 32)
  __nv_bfloat16 A2[16][kLd2];
  __nv_bfloat16 DZ1[16][kLd2];  // pre-activation gradients (rows x 32)
  __nv_bfloat16 DZ2[16][kLd2];
  __nv_bfloat16 DZ3[16][8];     // logit gradients (rows x o; 3..7 zero)
};

__device__ __forceinline__ uint32_t pair_of(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return uint32_t(__bfloat16_as_ushort(lo)) | (uint32_t(__bfloat16_as_ushort(hi)) << 16);
}

__device__ __forceinline__ void st32(__nv_bfloat16* p, uint32_t v) { *reinterpret_cast<uint32_t*>(p) = v; }

// A fragment of M^T for a [rows][cols] staged matrix M: m-index = column
// c0 + (g, g+8), k-index = row (2t.., 8+2t..).
template <int LD>
__device__ __forceinline__ void frag_t(const __nv_bfloat16 (*M)[LD], int c0, int g, int t, bool hi_rows_zero,
                                       uint32_t (&a)[4]) {
  a[0] = pair_of(M[2 * t][c0 + g], M[2 * t + 1][c0 + g]);
  a[2] = pair_of(M[8 + 2 * t][c0 + g], M[9 + 2 * t][c0 + g]);
  if (hi_rows_zero) {
    a[1] = 0u;
    a[3] = 0u;
  } else {
    a[1] = pair_of(M[2 * t][c0 + g + 8], M[2 * t + 1][c0 + g + 8]);
    a[3] = pair_of(M[8 + 2 * t][c0 + g + 8], M[9 + 2 * t][c0 + g + 8]);
  }
}

// B fragment of a [rows][cols] staged matrix M: k-index = row, n-index =
// column c0 + g.
template <int LD>
__device__ __forceinline__ void frag_b(const __nv_bfloat16 (*M)[LD], int c0, int g, int t, uint32_t& b0, uint32_t& b1) {
  b0 = pair_of(M[2 * t][c0 + g], M[2 * t + 1][c0 + g]);
  b1 = pair_of(M[8 + 2 * t][c0 + g], M[9 + 2 * t][c0 + g]);
}

__global__ void __launch_bounds__(32 * kGradWarps) mlp_grad_kernel(const MlpBlob* blob, const float* __restrict__ x,
                                                                   const float* __restrict__ y, long long n,
                                                                   float* __restrict__ grad, float* loss) {
  __shared__ MlpNet net;
  __shared__ __align__(16) __nv_bfloat16 W2T[32][kLd2];   // [in][out]
  __shared__ __align__(16) __nv_bfloat16 W3T[32][kLd1];   // [hidden][out], outputs 3.. zero
  __shared__ __align__(16) WarpStage stage[kGradWarps];
  __shared__ float gacc[kMlpParams];
  __shared__ float lacc;
  mlp_load_net(net, blob);
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) gacc[i] = 0.f;
  if (threadIdx.x == 0) lacc = 0.f;
  __syncthreads();
  for (int i = threadIdx.x; i < 32 * kLd2; i += blockDim.x) {
    const int r = i / kLd2, c = i - r * kLd2;   // r = in, c = out
    W2T[r][c] = c < 32 ? net.W2[c][r] : __float2bfloat16(0.f);
  }
  for (int i = threadIdx.x; i < 32 * kLd1; i += blockDim.x) {
    const int h = i / kLd1, o = i - h * kLd1;
    W3T[h][o] = o < 8 ? net.W3[o][h] : __float2bfloat16(0.f);
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, warp = threadIdx.x >> 5;
  WarpStage& S = stage[warp];
  MlpRegs R;
  mlp_load_regs(net, lane, R);
  const float sc = 2.f / float(n);
  float dW1[2][4] = {}, dW2[2][4][4] = {}, dW3[4][4] = {};
  float db1[4][2] = {}, db2[4][2] = {}, db3[3] = {};
  float lsum = 0.f;

  const long long groups = (n + 15) / 16;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long grp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; grp < groups; grp += nw) {
    const long long r0 = grp * 16 + g, r1 = r0 + 8;
    const bool ok0 = r0 < n, ok1 = r1 < n;
    const long long c0 = ok0 ? r0 : n - 1, c1 = ok1 ? r1 : n - 1;
    float v0[5], v1[5];
    load_stencil(x, c0, v0);
    load_stencil(x, c1, v1);
    float x0[5], x1[5];
    mlp_normalise(v0, x0);
    mlp_normalise(v1, x1);
    uint32_t xa[4];
    mlp_input_frag(x0, x1, t, xa);
    MlpCache f;
    float p0[3], p1[3];
    mlp_forward16(R, xa, f, p0, p1);

    // dL/dlogits through the softmax: dz3 = p (gp - <gp, p>), gp = 2(p - y)/n
    float dz3a[3], dz3b[3];
    {
      float gp0[3], gp1[3], s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float e0 = p0[k] - y[c0 * 3 + k], e1 = p1[k] - y[c1 * 3 + k];
        gp0[k] = ok0 ? sc * e0 : 0.f;
        gp1[k] = ok1 ? sc * e1 : 0.f;
        s0 = fmaf(gp0[k], p0[k], s0);
        s1 = fmaf(gp1[k], p1[k], s1);
        if (t == 0) lsum += (ok0 ? e0 * e0 : 0.f) + (ok1 ? e1 * e1 : 0.f);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        dz3a[k] = p0[k] * (gp0[k] - s0);
        dz3b[k] = p1[k] * (gp1[k] - s1);
        if (t == 0) db3[k] += dz3a[k] + dz3b[k];
      }
    }
    // da2 = dz3 W3 (K = outputs, padded to 16)
    uint32_t adz3[4];
    adz3[0] = pack_bf16(t == 0 ? dz3a[0] : (t == 1 ? dz3a[2] : 0.f), t == 0 ? dz3a[1] : 0.f);
    adz3[1] = pack_bf16(t == 0 ? dz3b[0] : (t == 1 ? dz3b[2] : 0.f), t == 0 ? dz3b[1] : 0.f);
    adz3[2] = 0u;
    adz3[3] = 0u;
    float dz2[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma16816(c, adz3, ld32(&W3T[nt * 8 + g][2 * t]), 0u);
#pragma unroll
      for (int i = 0; i < 4; ++i) dz2[nt][i] = c[i] * gelu_grad(f.z2[nt][i]);
      db2[nt][0] += dz2[nt][0] + dz2[nt][2];
      db2[nt][1] += dz2[nt][1] + dz2[nt][3];
    }
    // da1 = dz2 W2
    uint32_t adz2[2][4];
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      adz2[kk][0] = pack_bf16(dz2[2 * kk][0], dz2[2 * kk][1]);
      adz2[kk][1] = pack_bf16(dz2[2 * kk][2], dz2[2 * kk][3]);
      adz2[kk][2] = pack_bf16(dz2[2 * kk + 1][0], dz2[2 * kk + 1][1]);
      adz2[kk][3] = pack_bf16(dz2[2 * kk + 1][2], dz2[2 * kk + 1][3]);
    }
    float dz1[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
        mma16816(c, adz2[kk], ld32(&W2T[nt * 8 + g][16 * kk + 2 * t]), ld32(&W2T[nt * 8 + g][16 * kk + 8 + 2 * t]));
#pragma unroll
      for (int i = 0; i < 4; ++i) dz1[nt][i] = c[i] * gelu_grad(f.z1[nt][i]);
      db1[nt][0] += dz1[nt][0] + dz1[nt][2];
      db1[nt][1] += dz1[nt][1] + dz1[nt][3];
    }

    // stage the operands of the weight gradients
    if (t < 2) {
      const float* xs = t == 0 ? x0 : x1;
      const float* dz = t == 0 ? dz3a : dz3b;
      const int row = t == 0 ? g : g + 8;
#pragma unroll
      for (int j = 0; j < 8; ++j) S.X[row][j] = __float2bfloat16_rn(j < 5 ? xs[j] : 0.f);
#pragma unroll
      for (int k = 0; k < 8; ++k) S.DZ3[row][k] = __float2bfloat16_rn(k < 3 ? dz[k] : 0.f);
    }
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      st32(&S.A1[g][16 * kk + 2 * t], f.a1[kk][0]);
      st32(&S.A1[g + 8][16 * kk + 2 * t], f.a1[kk][1]);
      st32(&S.A1[g][16 * kk + 8 + 2 * t], f.a1[kk][2]);
      st32(&S.A1[g + 8][16 * kk + 8 + 2 * t], f.a1[kk][3]);
      st32(&S.A2[g][16 * kk + 2 * t], f.a2[kk][0]);
      st32(&S.A2[g + 8][16 * kk + 2 * t], f.a2[kk][1]);
      st32(&S.A2[g][16 * kk + 8 + 2 * t], f.a2[kk][2]);
      st32(&S.A2[g + 8][16 * kk + 8 + 2 * t], f.a2[kk][3]);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      st32(&S.DZ1[g][nt * 8 + 2 * t], pack_bf16(dz1[nt][0], dz1[nt][1]));
      st32(&S.DZ1[g + 8][nt * 8 + 2 * t], pack_bf16(dz1[nt][2], dz1[nt][3]));
      st32(&S.DZ2[g][nt * 8 + 2 * t], pack_bf16(dz2[nt][0], dz2[nt][1]));
      st32(&S.DZ2[g + 8][nt * 8 + 2 * t], pack_bf16(dz2[nt][2], dz2[nt][3]));
    }
    __syncwarp();
    // dW3 = dz3^T a2 (M = outputs, K = the 16 stencils, N = hidden)
    {
      uint32_t a[4];
      frag_t<8>(S.DZ3, 0, g, t, true, a);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        uint32_t b0, b1;
        frag_b<kLd2>(S.A2, nt * 8, g, t, b0, b1);
        mma16816(dW3[nt], a, b0, b1);
      }
    }
    // dW2 = dz2^T a1, dW1 = dz1^T x
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      uint32_t a[4];
      frag_t<kLd2>(S.DZ2, mt * 16, g, t, false, a);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        uint32_t b0, b1;
        frag_b<kLd2>(S.A1, nt * 8, g, t, b0, b1);
        mma16816(dW2[mt][nt], a, b0, b1);
      }
      frag_t<kLd2>(S.DZ1, mt * 16, g, t, false, a);
      uint32_t b0, b1;
      frag_b<8>(S.X, 0, g, t, b0, b1);
      mma16816(dW1[mt], a, b0, b1);
    }
    __syncwarp();
  }

  // reduce: registers -> CTA (shared atomics) -> global
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    if (g < 3) {
      atomicAdd(&gacc[kOffW3 + g * 32 + nt * 8 + 2 * t], dW3[nt][0]);
      atomicAdd(&gacc[kOffW3 + g * 32 + nt * 8 + 2 * t + 1], dW3[nt][1]);
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int o = mt * 16 + g, i = nt * 8 + 2 * t;
      atomicAdd(&gacc[kOffW2 + o * 32 + i], dW2[mt][nt][0]);
      atomicAdd(&gacc[kOffW2 + o * 32 + i + 1], dW2[mt][nt][1]);
      atomicAdd(&gacc[kOffW2 + (o + 8) * 32 + i], dW2[mt][nt][2]);
      atomicAdd(&gacc[kOffW2 + (o + 8) * 32 + i + 1], dW2[mt][nt][3]);
    }
    atomicAdd(&gacc[kOffB1 + nt * 8 + 2 * t], db1[nt][0]);
    atomicAdd(&gacc[kOffB1 + nt * 8 + 2 * t + 1], db1[nt][1]);
    atomicAdd(&gacc[kOffB2 + nt * 8 + 2 * t], db2[nt][0]);
    atomicAdd(&gacc[kOffB2 + nt * 8 + 2 * t + 1], db2[nt][1]);
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int o = mt * 16 + g;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * t + h;
      if (i < 5) {
        atomicAdd(&gacc[kOffW1 + o * 5 + i], dW1[mt][h]);
        atomicAdd(&gacc[kOffW1 + (o + 8) * 5 + i], dW1[mt][2 + h]);
      }
    }
  }
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) atomicAdd(&gacc[kOffB3 + k], db3[k]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) atomicAdd(&lacc, lsum);
  __syncthreads();
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) atomicAdd(&grad[i], gacc[i]);
  if (threadIdx.x == 0) atomicAdd(loss, lacc / float(n));
}

__global__ void mlp_harvest_kernel(const float* __restrict__ u, long long nx, long long ny,
                                   const long long* __restrict__ pos, long long count, int axis, int side, float d0,
                                   float d1, float d2, float* __restrict__ x, float* __restrict__ y, long long stride) {
  const float d[3] = {d0, d1, d2};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = pos[i];
    float v[5];
    if (p < 0 || p >= nx * ny) {
#pragma unroll
      for (int j = 0; j < 5; ++j) v[j] = __int_as_float(0x7fc00000);   // NaN marks a bad index
    } else {
      const long long xi = p % nx, yi = p / nx;
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        const long long o = side == 0 ? j - 3 : 3 - j;
        long long idx;
        if (axis == 0) {
          long long xx = (xi + o) % nx;
          if (xx < 0) xx += nx;
          idx = yi * nx + xx;
        } else {
          long long yy = (yi + o) % ny;
          if (yy < 0) yy += ny;
          idx = yy * nx + xi;
        }
        v[j] = u[idx];
      }
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) x[i * stride * 5 + j] = v[j];
    if (y) {
      float om[3];
      wenoz_omega(v, d, om);
#pragma unroll
      for (int r = 0; r < 3; ++r) y[i * stride * 3 + r] = om[r];
    }
  }
}

int grid_for(long long work, int block, int per_sm) {
  const long long cap = (long long)sm_count() * per_sm;
  long long g = (work + block - 1) / block;
  if (g > cap) g = cap;
  return int(g < 1 ? 1 : g);
}

molt_status launched() { return cudaGetLastError() == cudaSuccess ? MOLT_OK : MOLT_ECUDA; }

}  // namespace

extern "C" {

molt_status molt_weno_linear_weights(double nu, double* d) {
  if (!d || !(nu > 0) || !std::isfinite(nu)) return MOLT_EINVAL;
  QuadTable qt;
  if (!build_quadrature(5, nu, &qt)) return MOLT_EINVAL;
  for (int r = 0; r < 3; ++r) d[r] = qt.d[r];
  return MOLT_OK;
}

molt_status molt_quadrature_weights(int quad_points, double nu, double* c, double* sub, double* d) {
  if (!c || !(nu > 0) || !std::isfinite(nu)) return MOLT_EINVAL;
  QuadTable qt;
  if (!build_quadrature(quad_points, nu, &qt)) return MOLT_EINVAL;
  for (int i = 0; i < 6; ++i) c[i] = qt.c[i];
  for (int r = 0; r < 3; ++r) {
    for (int j = 0; j < 4; ++j)
      if (sub) sub[4 * r + j] = quad_points == 3 ? 0.0 : qt.sub[r][j];
    if (d) d[r] = quad_points == 3 ? 0.0 : qt.d[r];
  }
  return MOLT_OK;
}

molt_status molt_mlp_pack(const float* theta, void* blob, void* cuda_stream) {
  if (!theta || !blob || !aligned16(theta) || !aligned16(blob)) return MOLT_EINVAL;
  mlp_pack_kernel<<<1, 512, 0, static_cast<cudaStream_t>(cuda_stream)>>>(theta, static_cast<MlpBlob*>(blob));
  return launched();
}

molt_status molt_mlp_forward(const void* blob, const float* x, int64_t n, const double* d, float* w,
                             unsigned long long* fallbacks, void* cuda_stream) {
  if (n < 0 || !blob || !aligned16(blob)) return MOLT_EINVAL;
  if (n == 0) return MOLT_OK;
  if (!x || !w || !aligned16(x) || !aligned16(w)) return MOLT_EINVAL;
  const long long groups = (n + 15) / 16;
  const int grid = grid_for(groups * 32, 256, 8);
  mlp_forward_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      static_cast<const MlpBlob*>(blob), x, n, d ? float(d[0]) : 0.f, d ? float(d[1]) : 0.f, d ? float(d[2]) : 0.f,
      d ? 1 : 0, w, fallbacks);
  return launched();
}

molt_status molt_mlp_loss_grad(const void* blob, const float* x, const float* y, int64_t n, float* grad, float* loss,
                               void* cuda_stream) {
  if (n < 0 || !blob || !grad || !loss || !aligned16(blob) || !aligned16(grad)) return MOLT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s) != cudaSuccess ||
      cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess)
    return MOLT_ECUDA;
  if (n == 0) return MOLT_OK;
  if (!x || !y || !aligned16(x) || !aligned16(y)) return MOLT_EINVAL;
  const long long groups = (n + 15) / 16;
  const int grid = grid_for(groups * 32, 32 * kGradWarps, 8);
  mlp_grad_kernel<<<grid, 32 * kGradWarps, 0, s>>>(static_cast<const MlpBlob*>(blob), x, y, n, grad, loss);
  return launched();
}

molt_status molt_mlp_adam(float* theta, float* m, float* v, const float* grad, int64_t step, double lr, double beta1,
                          double beta2, double eps, void* blob, void* cuda_stream) {
  if (!theta || !m || !v || !grad || !blob || step < 1 || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) ||
      !(beta2 >= 0 && beta2 < 1) || !(eps > 0) || !aligned16(blob))
    return MOLT_EINVAL;
  const double bc1 = 1.0 - std::pow(beta1, double(step));
  const double bc2 = 1.0 - std::pow(beta2, double(step));
  mlp_adam_kernel<<<1, 512, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      theta, m, v, grad, float(lr), float(beta1), float(1.0 - beta1), float(beta2), float(1.0 - beta2), float(eps),
      float(bc1), float(bc2),
      static_cast<MlpBlob*>(blob));
  return launched();
}

molt_status molt_mlp_harvest(const float* u, int64_t nx, int64_t ny, const int64_t* pos, int64_t count, int axis,
                             int side, const double* d, float* x, float* y, int64_t stride, void* cuda_stream) {
  if (count < 0 || nx < 1 || ny < 1 || (axis != 0 && axis != 1) || (side != 0 && side != 1) || stride < 1)
    return MOLT_EINVAL;
  if (count == 0) return MOLT_OK;
  if (!u || !pos || !x || (y && !d)) return MOLT_EINVAL;
  const int grid = grid_for(count, 256, 8);
  mlp_harvest_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      u, nx, ny, reinterpret_cast<const long long*>(pos), count, axis, side, d ? float(d[0]) : 0.f,
      d ? float(d[1]) : 0.f, d ? float(d[2]) : 0.f, x, y, stride);
  return launched();
}

}  // extern "C"

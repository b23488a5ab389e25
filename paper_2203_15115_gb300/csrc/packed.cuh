// Packed FP32 arithmetic (two lanes of a float2 per instruction: FADD2,
// FFMA2, FMUL2 of sm_100+), 4-byte asynchronous global -> shared copies, and
// the modal element forces of afd_common.cuh in packed form.  Shared by the
// FP32 stencils (Sec. 3.5: the operator apply is the cost of an iteration).
#pragma once

#include "afd_common.cuh"

namespace afd {

__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, rounded once (b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Asynchronous global -> shared copies of 4 bytes (cp.async, sm_80+), used to
// stage node values a few planes ahead without holding registers.  With
// valid = false nothing is read and the destination is zero-filled (the
// source operand must still be a mapped address).
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gmem_src, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem_src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Modal forces of two elements (modal_forces in afd_common.cuh, lane-wise),
// h[c][0] (the rigid translation) is neither read nor written.
__device__ __forceinline__ void modal_forces2(float2 (&h)[3][8], float2 E, const ElemConsts<float>& K) {
  const float2 l16 = mul2(bc2(K.l16), E), m16 = mul2(bc2(K.m16), E), m8 = mul2(bc2(K.m8), E);
  const float2 l48 = mul2(bc2(K.l48), E), m48 = mul2(bc2(K.m48), E), m3 = mul2(bc2(K.m3_48), E);
  const float2 t144 = mul2(bc2(K.t144), E);
  {
    const float2 Axx = h[0][1], Ayy = h[1][2], Azz = h[2][4];
    const float2 tr = mul2(l16, add2(add2(Axx, Ayy), Azz));
    const float2 sxy = mul2(m16, add2(h[0][2], h[1][1]));
    const float2 syz = mul2(m16, add2(h[1][4], h[2][2]));
    const float2 szx = mul2(m16, add2(h[2][1], h[0][4]));
    h[0][1] = fma2(m8, Axx, tr);
    h[1][2] = fma2(m8, Ayy, tr);
    h[2][4] = fma2(m8, Azz, tr);
    h[0][2] = sxy; h[1][1] = sxy;
    h[1][4] = syz; h[2][2] = syz;
    h[2][1] = szx; h[0][4] = szx;
  }
  {
    const float2 Px = h[0][3], Py = h[1][3], Pz = h[2][3];
    const float2 Qx = h[0][6], Qy = h[1][6], Qz = h[2][6];
    const float2 Rx = h[0][5], Ry = h[1][5], Rz = h[2][5];
    const float2 s1 = mul2(l48, add2(Px, Qz));
    const float2 s2 = mul2(l48, add2(Py, Rz));
    const float2 s3 = mul2(l48, add2(Rx, Qy));
    const float2 s = add2(add2(Pz, Qx), Ry);
    h[0][3] = fma2(m3, Px, s1);
    h[2][6] = fma2(m3, Qz, s1);
    h[1][3] = fma2(m3, Py, s2);
    h[2][5] = fma2(m3, Rz, s2);
    h[0][5] = fma2(m3, Rx, s3);
    h[1][6] = fma2(m3, Qy, s3);
    h[2][3] = mul2(m48, add2(Pz, s));
    h[0][6] = mul2(m48, add2(Qx, s));
    h[1][5] = mul2(m48, add2(Ry, s));
  }
  h[0][7] = mul2(h[0][7], t144);
  h[1][7] = mul2(h[1][7], t144);
  h[2][7] = mul2(h[2][7], t144);
}

}  // namespace afd

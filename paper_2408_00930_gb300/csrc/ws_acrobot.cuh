// ws_acrobot.cuh -- the acrobot's physics in FP32, shared by the per-step
// kernel (ws_plain.cu) and the fused tensor-core kernel (ws_control_tc.cu).
#pragma once

#include <math.h>

namespace ws {

// sin / cos for the physics.  FAST (the fused BF16 kernels): the SFU's
// approximate sin and cos after reducing the argument to [-pi, pi] with
// x - 2 pi rint(x / 2 pi), and approximate divisions; else CUDA's accurate
// functions and IEEE division (the FP32 paths).
template <bool FAST>
__device__ __forceinline__ void acro_sincos(float x, float *s, float *c) {
  if (FAST) {
    const float r = fmaf(-6.28318530717959f, rintf(x * 0.159154943091895f), x);
    *s = __sinf(r);
    *c = __cosf(r);
  } else {
    sincosf(x, s, c);
  }
}
template <bool FAST>
__device__ __forceinline__ float acro_sin(float x) {
  if (FAST) return __sinf(fmaf(-6.28318530717959f, rintf(x * 0.159154943091895f), x));
  return sinf(x);
}
template <bool FAST>
__device__ __forceinline__ float acro_cos(float x) {
  if (FAST) return __cosf(fmaf(-6.28318530717959f, rintf(x * 0.159154943091895f), x));
  return cosf(x);
}

// a / b: FAST the approximate division (two ulp, the SFU's reciprocal and one
// product); else IEEE division.
template <bool FAST>
__device__ __forceinline__ float acro_div(float a, float b) {
  return FAST ? __fdividef(a, b) : a / b;
}

// Two-link acrobot of Sutton & Barto (paper App. C, classic control), book
// dynamics: m1 = m2 = l1 = I1 = I2 = 1, lc1 = lc2 = 0.5, g = 9.8, angles from
// hanging down, torque tau on the second joint.
template <bool FAST>
__device__ __forceinline__ void acro_accel(float th1, float th2, float w1, float w2, float tau,
                                           float &acc1, float &acc2) {
  const float m1 = 1.f, m2 = 1.f, l1 = 1.f, lc1 = 0.5f, lc2 = 0.5f, I1 = 1.f, I2 = 1.f, g = 9.8f;
  float s2, c2;
  acro_sincos<FAST>(th2, &s2, &c2);
  const float d1 = m1 * lc1 * lc1 + m2 * (l1 * l1 + lc2 * lc2 + 2.f * l1 * lc2 * c2) + I1 + I2;
  const float d2 = m2 * (lc2 * lc2 + l1 * lc2 * c2) + I2;
  const float phi2 = m2 * lc2 * g * acro_sin<FAST>(th1 + th2);
  const float phi1 = -m2 * l1 * lc2 * w2 * w2 * s2 - 2.f * m2 * l1 * lc2 * w2 * w1 * s2 +
                     (m1 * lc1 + m2 * l1) * g * acro_sin<FAST>(th1) + phi2;
  acc2 = acro_div<FAST>(tau + acro_div<FAST>(d2, d1) * phi1 - m2 * l1 * lc2 * w1 * w1 * s2 - phi2,
                        m2 * lc2 * lc2 + I2 - acro_div<FAST>(d2 * d2, d1));
  acc1 = acro_div<FAST>(-(d2 * acc2 + phi1), d1);
}

// One classic RK4 step of dt with tau held; angles wrapped into [-pi, pi],
// velocities clipped to |w1| <= 4 pi, |w2| <= 9 pi.
template <bool FAST>
__device__ __forceinline__ void acro_step(float (&s)[4], float tau, float dt) {
  float k[4][4];
  float y[4] = {s[0], s[1], s[2], s[3]};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    k[q][0] = y[2];
    k[q][1] = y[3];
    acro_accel<FAST>(y[0], y[1], y[2], y[3], tau, k[q][2], k[q][3]);
    if (q < 3) {
      const float h = q < 2 ? 0.5f * dt : dt;
#pragma unroll
      for (int i = 0; i < 4; ++i) y[i] = s[i] + h * k[q][i];
    }
  }
  const float kPi = 3.14159265358979f, k2Pi = 6.28318530717959f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    s[i] = s[i] + dt / 6.f * (k[0][i] + 2.f * k[1][i] + 2.f * k[2][i] + k[3][i]);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    for (int it = 0; it < 64 && s[i] > kPi; ++it) s[i] -= k2Pi;
    for (int it = 0; it < 64 && s[i] < -kPi; ++it) s[i] += k2Pi;
  }
  s[2] = fminf(fmaxf(s[2], -4.f * kPi), 4.f * kPi);
  s[3] = fminf(fmaxf(s[3], -9.f * kPi), 9.f * kPi);
}

// Tip height above the pivot in link lengths; terminal above 1.
template <bool FAST>
__device__ __forceinline__ bool acro_terminal(const float (&s)[4]) {
  return -acro_cos<FAST>(s[0]) - acro_cos<FAST>(s[0] + s[1]) > 1.0f;
}

}  // namespace ws

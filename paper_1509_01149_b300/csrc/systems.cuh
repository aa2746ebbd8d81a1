// The three plants of the MPPI workloads and their state costs, FP32 device code.
//
// Each model provides N (state size), M (control size), an Aux register block,
//   init(x, aux, env)          -- set up per-sample auxiliaries at x0
//   step(x, v, aux, env, dt)   -- advance the state under control v = u_i + du_i
//   cost(x, aux, env)          -- running state cost q at the current state
// The terminal cost phi is q of the final state.
//
// Models (the paper's own car and quadrotor models come from external works;
// these are the synthetic stand-ins of the workloads):
//   CartPole  force input, pole-on-cart with a uniform rod of half-length l,
//             explicit Euler (Sec. II-A); q = x^2 + xdot^2 + 10 theta^2 + thetadot^2.
//   Car       dynamic bicycle, first-order steering actuator, simplified Pacejka
//             tyres D sin(C atan(B alpha)); explicit Euler (position and heading sums
//             Kahan-compensated); q = bilinear cost-map lookup + (vx - 7)^2 (speed
//             term of Sec. V-B).
//   Quad      12-state rigid body, four rotor thrusts in a "+" layout, ZYX Euler
//             angles, RK4; q of Sec. V-C with crash weight 1e4.  A crash (cylinder,
//             ground, |pitch| >= 1.4 rad or a non-finite step) stops the rollout: the
//             state stays at the last valid state and the crash cost keeps accruing.
#pragma once
#include "mppi_device.cuh"

namespace mppi {

struct Env {
  const float *__restrict__ map;
  int map_w, map_h;
  float map_ox, map_oy, map_inv_cell;
  const float *obs;  // cylinders: [n_obs][4] (cx, cy, r, 0) in shared memory when obs_packed,
                     // else [n_obs][3] in global memory
  int n_obs;
  int obs_packed;
  float gx, gy, gz;
  // nearest-cylinder grid in shared memory (with obs_packed; grid_nx == 0: none): per cell the
  // list of cylinders that can be nearest to a point of the cell (see forest_grid.h)
  const unsigned short *grid_off;  // [grid_nx * grid_ny + 1] list starts in grid_idx
  const unsigned char *grid_idx;
  int grid_nx, grid_ny;
  float grid_ox, grid_oy, grid_inv_h;
};

// ---------------------------------------------------------------------------
// sin and cos of an unbounded angle: reduced to [-pi, pi] by the two-constant Cody-Waite
// scheme (k = nearest integer to a / 2 pi; a - k hi - k lo with hi + lo = 2 pi, hi the nearest
// float), then both on the special-function unit (about 2^-21 absolute on the reduced range).
// No slow-path branch, so consecutive steps interleave.
__device__ __forceinline__ void sincos_reduced(float a, float &s, float &c) {
  constexpr float two_pi_hi = 6.28318548202514648f;
  constexpr float two_pi_lo = -1.7484556025237907e-07f;
  constexpr float inv_two_pi = 0.159154943091895336f;
  const float kk = rintf(a * inv_two_pi);
  float red = fmaf(-kk, two_pi_hi, a);
  red = fmaf(-kk, two_pi_lo, red);
  __sincosf(red, &s, &c);
}

struct CartPole {
  static constexpr int N = 4, M = 1;
  struct Aux {};
  static constexpr float mc = 1.0f, mp = 0.1f, l = 0.5f, g = 9.81f;

  __device__ __forceinline__ static void init(const float *, Aux &, const Env &) {}

  __device__ __forceinline__ static void step(float x[N], const float v[M], Aux &, const Env &, float dt) {
    constexpr float inv_Mt = 1.0f / (mc + mp);
    float s, c;
    sincos_reduced(x[2], s, c);
    const float tmp = (v[0] + mp * l * x[3] * x[3] * s) * inv_Mt;
    const float th_acc = __fdividef(g * s - c * tmp, l * (4.0f / 3.0f - mp * c * c * inv_Mt));
    const float x_acc = tmp - mp * l * th_acc * c * inv_Mt;
    x[0] += dt * x[1];
    x[1] += dt * x_acc;
    x[2] += dt * x[3];
    x[3] += dt * th_acc;
  }

  __device__ __forceinline__ static float cost(const float x[N], const Aux &, const Env &) {
    return x[0] * x[0] + x[1] * x[1] + 10.0f * x[2] * x[2] + x[3] * x[3];
  }

  // cost in two halves (see Car): nothing to load here
  struct Pending {
    float q;
  };
  __device__ __forceinline__ static Pending cost_issue(const float x[N], const Aux &a, const Env &e) {
    return Pending{cost(x, a, e)};
  }
  __device__ __forceinline__ static float cost_finish(const Pending &pd, const Env &) { return pd.q; }
};

// ---------------------------------------------------------------------------
// The cart-pole of Sec. V-A: the control is a desired cart velocity, p'' = 10 (u - p');
// the pole is a uniform rod of half-length l with theta = 0 hanging down,
// theta'' = -(3 / (4 l)) (g sin theta + p'' cos theta); explicit Euler.
// q = p^2 + 500 (1 + cos theta)^2 + theta'^2 + p'^2.
struct CartPoleVel {
  static constexpr int N = 4, M = 1;
  struct Aux {};
  static constexpr float l = 0.5f, g = 9.81f, k_vel = 10.0f;

  __device__ __forceinline__ static void init(const float *, Aux &, const Env &) {}

  __device__ __forceinline__ static void step(float x[N], const float v[M], Aux &, const Env &, float dt) {
    float s, c;
    sincos_reduced(x[2], s, c);
    const float acc = k_vel * (v[0] - x[1]);
    const float th_acc = -(3.0f / (4.0f * l)) * (g * s + acc * c);
    x[0] += dt * x[1];
    x[1] += dt * acc;
    x[2] += dt * x[3];
    x[3] += dt * th_acc;
  }

  __device__ __forceinline__ static float cost(const float x[N], const Aux &, const Env &) {
    float s, c;
    sincos_reduced(x[2], s, c);
    const float up = 1.0f + c;
    return x[0] * x[0] + 500.0f * up * up + x[3] * x[3] + x[1] * x[1];
  }

  struct Pending {
    float q;
  };
  __device__ __forceinline__ static Pending cost_issue(const float x[N], const Aux &a, const Env &e) {
    return Pending{cost(x, a, e)};
  }
  __device__ __forceinline__ static float cost_finish(const Pending &pd, const Env &) { return pd.q; }
};

// ---------------------------------------------------------------------------
// +-0 for a finite position, NaN for a non-finite one.  The cost map has no value at a
// non-finite position: adding this to the map term makes the sample's cost NaN (weight 0)
// instead of the clamped edge value, and leaves every finite cost unchanged to the bit.
__device__ __forceinline__ float position_nan(float X, float Y) { return fmaf(Y, 0.0f, X * 0.0f); }

// Bilinear lookup of a cost map [H][W], node (ix, iy) at (ox + ix/inv_cell, oy + iy/inv_cell),
// finite coordinates clamped to the grid; NaN at a non-finite coordinate.
__device__ __forceinline__ float map_bilinear(const Env &e, float X, float Y) {
  const float fx = fminf(fmaxf((X - e.map_ox) * e.map_inv_cell, 0.0f), static_cast<float>(e.map_w - 1));
  const float fy = fminf(fmaxf((Y - e.map_oy) * e.map_inv_cell, 0.0f), static_cast<float>(e.map_h - 1));
  const int ix = min(static_cast<int>(fx), e.map_w - 2);
  const int iy = min(static_cast<int>(fy), e.map_h - 2);
  const float tx = fx - static_cast<float>(ix);
  const float ty = fy - static_cast<float>(iy);
  const float *row = e.map + static_cast<size_t>(iy) * e.map_w + ix;
  const float m00 = __ldg(row), m10 = __ldg(row + 1);
  const float m01 = __ldg(row + e.map_w), m11 = __ldg(row + e.map_w + 1);
  const float a = m00 + tx * (m10 - m00);
  const float b = m01 + tx * (m11 - m01);
  return (a + ty * (b - a)) + position_nan(X, Y);
}

struct Car {
  static constexpr int N = 7, M = 2;
  // Compensation terms of the three states that accumulate without bound (X, Y, psi):
  // their Euler sums are Kahan-compensated so that FP32 rounding of a large position
  // does not drift along the horizon.
  struct Aux {
    float cX, cY, cpsi;
  };
  static constexpr float m = 21.7f, Iz = 1.12f, lf = 0.34f, lr = 0.23f;
  static constexpr float B = 4.0f, C = 1.8f, mu = 0.9f, g = 9.81f;
  static constexpr float delta_max = 0.5f, tau_delta = 0.1f;
  static constexpr float Cm = 120.0f, Crr = 2.0f, Cd = 0.35f, vx_floor = 1.0f, v_target = 7.0f;
  static constexpr float Df = mu * m * g * lr / (lf + lr);
  static constexpr float Dr = mu * m * g * lf / (lf + lr);

  __device__ __forceinline__ static void init(const float *, Aux &a, const Env &) { a.cX = a.cY = a.cpsi = 0.0f; }

  // The step splits into the velocity recurrence (vx, vy, r, delta), which depends only on
  // itself and the control, and the pose rates (X, Y, psi), which read the velocities but
  // never feed back into them.
  //
  // The shape sin(C atan z), z = B alpha, is evaluated on the whole real line through
  // v = |z| / (1 + |z|) in [0, 1], where it is analytic: sign(z) v P(v) / Q(v), a rational
  // fitted towards minimax (maximum absolute error 3.0e-7 in exact arithmetic, ~6.5e-7 in
  // FP32; tyre_shape_fit.py prints the coefficients).  Two reciprocals and ten FMAs with no
  // branch replace an arctangent and a sine on the recurrence's critical path.  |z| is capped
  // at 1e30 (the shape equals its limit sin(C pi / 2) there to FP32 precision; the cap keeps
  // the fast reciprocal in range); NaN propagates.
  __device__ __forceinline__ static float tyre_shape(float z) {
    const float a = fabsf(z) > 1.0e30f ? 1.0e30f : fabsf(z);
    const float v = __fdividef(a, 1.0f + a);
    float P = -1.802042631e+00f;
    P = fmaf(P, v, 2.115236191e+00f);
    P = fmaf(P, v, 2.735651234e-01f);
    P = fmaf(P, v, -1.707349900e+00f);
    P = fmaf(P, v, 1.799983406e+00f);
    float Q = 2.216846433e+00f;
    Q = fmaf(Q, v, -2.120366621e+00f);
    Q = fmaf(Q, v, 1.076769485e+00f);
    Q = fmaf(Q, v, 1.973980183e+00f);
    Q = fmaf(Q, v, -1.948672322e+00f);
    Q = fmaf(Q, v, 1.000000000e+00f);
    return copysignf(__fdividef(v * P, Q), z);
  }
  // The same force as a function of t = tan(alpha) = n / d (d > 0, so |alpha| < pi/2):
  // sin(C atan(B atan t)) = sign(n) v P(v) / Q(v) with v = |t| / (1 + |t|) = |n| / (|n| + d),
  // P and Q of degree 6 fitted like tyre_shape (maximum error 2.5e-7 in exact arithmetic,
  // ~4.5e-7 in FP32; tyre_shape_fit.py prints the coefficients).  Given the slip angle as a
  // ratio, no arctangent and no reciprocal of the speed are needed.
  __device__ __forceinline__ static float slip_shape(float n, float d) {
    const float an = fabsf(n);
    const float v = __fdividef(an, an + d);
    float P = 8.201814610e+00f;
    P = fmaf(P, v, 6.672181936e+01f);
    P = fmaf(P, v, 3.717660575e+01f);
    P = fmaf(P, v, 4.971201143e+00f);
    P = fmaf(P, v, 2.782720545e+01f);
    P = fmaf(P, v, 1.013812583e+01f);
    P = fmaf(P, v, 7.200033913e+00f);
    float Q = 2.088930100e+02f;
    Q = fmaf(Q, v, -5.017322148e+01f);
    Q = fmaf(Q, v, 8.035395784e+01f);
    Q = fmaf(Q, v, 3.080427926e+01f);
    Q = fmaf(Q, v, 1.677532802e+01f);
    Q = fmaf(Q, v, 4.081411398e-01f);
    Q = fmaf(Q, v, 1.000000000e+00f);
    return copysignf(__fdividef(v * P, Q), n);
  }
  // The shape sin(C atan(B theta)) of a slip angle of magnitude theta in [0, pi] given as a
  // direction (n, d), a positive multiple of (sin alpha, cos alpha), signed like n.  Through the
  // half-angle tangent tau = tan(theta / 2) = |n| / (rho + d) = (rho - d) / |n|, rho = |(n, d)|
  // (the first form for d >= 0, the second for d < 0: neither cancels),
  // v = tau / (1 + tau) = num / (|n| + rho + |d|), and v P(v) / Q(v) with P and Q of degree 7
  // fitted like tyre_shape (maximum error 3.5e-8 in exact arithmetic, ~2.7e-7 in FP32;
  // tyre_shape_fit.py prints the coefficients).  One square root and two reciprocals on the
  // special-function unit, no arctangent.  (n, d) is finite and not (0, 0).
  __device__ __forceinline__ static float angle_shape(float n, float d) {
    const float an = fabsf(n), ad = fabsf(d);
    const float q = fmaf(n, n, d * d);
    const float rho = q * rsqrtf(q);
    const float num = d >= 0.0f ? an : rho + ad;
    const float v = __fdividef(num, (an + rho) + ad);
    float P = -8.540411824e+01f;
    P = fmaf(P, v, 1.562593909e+03f);
    P = fmaf(P, v, -4.858328297e+02f);
    P = fmaf(P, v, 1.212054441e+03f);
    P = fmaf(P, v, -4.118799750e+02f);
    P = fmaf(P, v, 5.340800569e+02f);
    P = fmaf(P, v, 2.681955798e+01f);
    P = fmaf(P, v, 1.439997149e+01f);
    float Q = 2.627731536e+03f;
    Q = fmaf(Q, v, 1.923390719e+03f);
    Q = fmaf(Q, v, -1.496429105e+03f);
    Q = fmaf(Q, v, 2.121401013e+03f);
    Q = fmaf(Q, v, 9.330799874e+01f);
    Q = fmaf(Q, v, 9.149840455e+01f);
    Q = fmaf(Q, v, 8.619579532e-01f);
    Q = fmaf(Q, v, 1.000000000e+00f);
    return copysignf(__fdividef(v * P, Q), n);
  }
  // Velocity rates from the two lateral forces (shared by both step forms below).
  __device__ __forceinline__ static void vel_rates(float vx, float vy, float r, float delta, const float v[M],
                                                   float Fyf, float Fyr, float sd, float cd, float d[4]) {
    const float Fx = Cm * v[1] - Crr * vx - Cd * vx * fabsf(vx);
    d[0] = (Fx - Fyf * sd) * (1.0f / m) + vy * r;
    d[1] = (Fyr + Fyf * cd) * (1.0f / m) - vx * r;
    d[2] = (lf * Fyf * cd - lr * Fyr) * (1.0f / Iz);
    d[3] = (delta_max * v[0] - delta) * (1.0f / tau_delta);
  }
  // The steering angle's sine and cosine run on the special-function unit (about 2^-21
  // absolute for |delta| < pi), as single operations with no slow-path branch.
  __device__ __forceinline__ static void deriv_vel(float vx, float vy, float r, float delta, const float v[M],
                                                   float d[4]) {
    const float inv_vxs = __fdividef(1.0f, fmaxf(vx, vx_floor));
    const float alpha_f = delta - atanf((vy + lf * r) * inv_vxs);
    const float alpha_r = -atanf((vy - lr * r) * inv_vxs);
    float sd, cd;
    __sincosf(delta, &sd, &cd);
    vel_rates(vx, vy, r, delta, v, Df * tyre_shape(B * alpha_f), Dr * tyre_shape(B * alpha_r), sd, cd, d);
  }
  // The same rates with no arctangent and no reciprocal of the speed on the recurrence's
  // critical path.  Rear: alpha_r = -atan((vy - lr r) / vxs), so tan(alpha_r) =
  // (lr r - vy) / vxs with vxs >= 1 > 0 (slip_shape).  Front: alpha_f = delta - phi,
  // phi = atan(w / vxs) in (-pi/2, pi/2), w = vy + lf r; by the angle difference
  // (n, d) = (vxs sin(delta) - w cos(delta), vxs cos(delta) + w sin(delta)) is a positive
  // multiple of (sin alpha_f, cos alpha_f), so angle_shape(n, d) is the force of the angle
  // wrapped into [-pi, pi].  That is alpha_f itself when |delta| < 1.5 (< pi/2, so
  // |alpha_f| < pi), and when |delta| < 3 (< pi, so |alpha_f| < 3 pi/2) with n of delta's
  // sign (alpha_f in (delta - pi/2, delta + pi/2) wraps only past +-pi, which flips the sign
  // of n).  Returns false outside that domain (a slip angle past +-pi, a steering angle of
  // 3 rad or more, or a NaN), where the rates are not valid and the caller takes deriv_vel.
  __device__ __forceinline__ static bool deriv_vel_ratio(float vx, float vy, float r, float delta, const float v[M],
                                                         float d[4]) {
    const float vxs = fmaxf(vx, vx_floor);
    float sd, cd;
    __sincosf(delta, &sd, &cd);
    const float w = fmaf(lf, r, vy);
    const float nf = fmaf(sd, vxs, -(w * cd));
    const float df = fmaf(cd, vxs, w * sd);
    vel_rates(vx, vy, r, delta, v, Df * angle_shape(nf, df), Dr * slip_shape(fmaf(lr, r, -vy), vxs), sd, cd, d);
    const float ad = fabsf(delta);
    return ad < 1.5f || (ad < 3.0f && nf * delta > 0.0f);
  }
  // The heading is unbounded: sincos_reduced (Cody-Waite reduction, then the SFU).
  __device__ __forceinline__ static void sincos_heading(float psi, float &s, float &c) { sincos_reduced(psi, s, c); }
  __device__ __forceinline__ static void pose_rates(float psi, float vx, float vy, float &dX, float &dY) {
    float sp, cp;
    sincos_heading(psi, sp, cp);
    dX = vx * cp - vy * sp;
    dY = vx * sp + vy * cp;
  }

  __device__ __forceinline__ static void deriv(const float x[N], const float v[M], float d[N]) {
    pose_rates(x[2], x[3], x[4], d[0], d[1]);
    d[2] = x[5];
    deriv_vel(x[3], x[4], x[5], x[6], v, d + 3);
  }

  // x += h with the running compensation c (Kahan): keeps the rounding of x out of the sum.
  __device__ __forceinline__ static void comp_add(float &x, float &c, float h) {
    const float y = h - c;
    const float t = x + y;
    c = (t - x) - y;
    x = t;
  }

  __device__ __forceinline__ static void step(float x[N], const float v[M], Aux &a, const Env &, float dt) {
    float d[N];
    deriv(x, v, d);
    comp_add(x[0], a.cX, dt * d[0]);
    comp_add(x[1], a.cY, dt * d[1]);
    comp_add(x[2], a.cpsi, dt * d[2]);
#pragma unroll
    for (int i = 3; i < N; ++i) x[i] += dt * d[i];
  }
  // The two halves of step() on their own (same arithmetic): xv = (vx, vy, r, delta).
  __device__ __forceinline__ static void vel_step(float xv[4], const float v[M], float dt) {
    float d[4];
    deriv_vel(xv[0], xv[1], xv[2], xv[3], v, d);
#pragma unroll
    for (int i = 0; i < 4; ++i) xv[i] += dt * d[i];
  }
  // vel_step through deriv_vel_ratio; false (xv not valid) outside the ratio's domain.
  __device__ __forceinline__ static bool vel_step_ratio(float xv[4], const float v[M], float dt) {
    float d[4];
    const bool in = deriv_vel_ratio(xv[0], xv[1], xv[2], xv[3], v, d);
#pragma unroll
    for (int i = 0; i < 4; ++i) xv[i] += dt * d[i];
    return in;
  }
  // pose (X, Y, psi) over one step from the velocities (vx, vy, r) at the step's start
  __device__ __forceinline__ static void pose_step(float &X, float &Y, float &psi, Aux &a, float vx, float vy, float r,
                                                   float dt) {
    float dX, dY;
    pose_rates(psi, vx, vy, dX, dY);
    comp_add(X, a.cX, dt * dX);
    comp_add(Y, a.cY, dt * dY);
    comp_add(psi, a.cpsi, dt * r);
  }

  __device__ __forceinline__ static float cost(const float x[N], const Aux &, const Env &e) {
    const float dv = x[3] - v_target;
    return map_bilinear(e, x[0], x[1]) + dv * dv;
  }

  // The cost in two halves: cost_issue starts the four map loads of q(x) and returns at
  // once; cost_finish combines them.  The rollout finishes step i's cost only after the
  // dynamics of step i+1, so the L2 latency of the loads overlaps a step of arithmetic.
  struct Pending {
    float m00, m10, m01, m11, tx, ty, speed;
  };
  __device__ __forceinline__ static Pending cost_issue(const float x[N], const Aux &, const Env &e) {
    Pending pd;
    const float fx = fminf(fmaxf((x[0] - e.map_ox) * e.map_inv_cell, 0.0f), static_cast<float>(e.map_w - 1));
    const float fy = fminf(fmaxf((x[1] - e.map_oy) * e.map_inv_cell, 0.0f), static_cast<float>(e.map_h - 1));
    const int ix = min(static_cast<int>(fx), e.map_w - 2);
    const int iy = min(static_cast<int>(fy), e.map_h - 2);
    pd.tx = fx - static_cast<float>(ix);
    pd.ty = fy - static_cast<float>(iy);
    const float *row = e.map + static_cast<size_t>(iy) * e.map_w + ix;
    pd.m00 = __ldg(row);
    pd.m10 = __ldg(row + 1);
    pd.m01 = __ldg(row + e.map_w);
    pd.m11 = __ldg(row + e.map_w + 1);
    const float dv = x[3] - v_target;
    pd.speed = fmaf(dv, dv, position_nan(x[0], x[1]));
    return pd;
  }
  __device__ __forceinline__ static float cost_finish(const Pending &pd, const Env &) {
    const float a = pd.m00 + pd.tx * (pd.m10 - pd.m00);
    const float b = pd.m01 + pd.tx * (pd.m11 - pd.m01);
    return (a + pd.ty * (b - a)) + pd.speed;
  }
};

// ---------------------------------------------------------------------------
struct Quad {
  static constexpr int N = 12, M = 4;
  struct Aux {
    float d;       // obstacle distance at the current state
    bool crashed;
  };
  static constexpr float mass = 0.5f, g = 9.81f, arm = 0.17f, kappa = 0.016f;
  static constexpr float Ixx = 2.3e-3f, Iyy = 2.3e-3f, Izz = 4.0e-3f, pitch_limit = 1.4f;
  static constexpr float w_xy = 2.5f, w_z = 150.0f, w_yaw = 50.0f, w_v = 1.0f;
  static constexpr float w_obs = 350.0f, obs_scale = 12.0f, w_crash = 1.0e4f;

  // The quadrotor path uses the hardware-approximate elementary functions (sincos,
  // reciprocal square root, exp): its path costs stay within ~1e-6 of the FP64 oracle,
  // far inside the 1e-4 bar, and these functions are most of its instructions.
  __device__ __forceinline__ static float fast_sqrt(float a) {
    const float s = fmaxf(a, 1e-30f);
    return s * rsqrtf(s);
  }

  // Nearest cylinder surface.  The minimum is exact in any order, so the packed path keeps
  // four independent running minima (a 4-wide dependency chain instead of one of n_obs).
  __device__ __forceinline__ static float obstacle_distance(const Env &e, float px, float py) {
    float d = INFINITY;
    if (e.obs_packed) {  // one 128-bit broadcast load per cylinder
      const float4 *o4 = reinterpret_cast<const float4 *>(e.obs);
      float d0 = INFINITY, d1 = INFINITY, d2 = INFINITY, d3 = INFINITY;
      int j = 0;
#pragma unroll 2
      for (; j + 3 < e.n_obs; j += 4) {
        const float4 c0 = o4[j], c1 = o4[j + 1], c2 = o4[j + 2], c3 = o4[j + 3];
        float ax = px - c0.x, ay = py - c0.y;
        d0 = fminf(d0, fast_sqrt(fmaf(ax, ax, ay * ay)) - c0.z);
        ax = px - c1.x, ay = py - c1.y;
        d1 = fminf(d1, fast_sqrt(fmaf(ax, ax, ay * ay)) - c1.z);
        ax = px - c2.x, ay = py - c2.y;
        d2 = fminf(d2, fast_sqrt(fmaf(ax, ax, ay * ay)) - c2.z);
        ax = px - c3.x, ay = py - c3.y;
        d3 = fminf(d3, fast_sqrt(fmaf(ax, ax, ay * ay)) - c3.z);
      }
      for (; j < e.n_obs; ++j) {
        const float4 c = o4[j];
        const float ax = px - c.x, ay = py - c.y;
        d0 = fminf(d0, fast_sqrt(fmaf(ax, ax, ay * ay)) - c.z);
      }
      d = fminf(fminf(d0, d1), fminf(d2, d3));
    } else {
#pragma unroll 4
      for (int j = 0; j < e.n_obs; ++j) {
        const float dx = px - e.obs[3 * j], dy = py - e.obs[3 * j + 1];
        d = fminf(d, fast_sqrt(fmaf(dx, dx, dy * dy)) - e.obs[3 * j + 2]);
      }
    }
    return d;
  }

  // The same minimum split over a group of `lanes` consecutive lanes that hold the same
  // sample (lane s takes cylinders s, s + lanes, ...), combined by butterfly shuffles.  Every
  // lane of the warp must call it together; obstacles packed as float4.
  __device__ __forceinline__ static float obstacle_distance_lanes(const Env &e, float px, float py, int sub,
                                                                  int lanes) {
    const float4 *o4 = reinterpret_cast<const float4 *>(e.obs);
    float d0 = INFINITY, d1 = INFINITY;
    int j = sub;
    for (; j + lanes < e.n_obs; j += 2 * lanes) {
      const float4 c0 = o4[j], c1 = o4[j + lanes];
      float ax = px - c0.x, ay = py - c0.y;
      d0 = fminf(d0, fast_sqrt(fmaf(ax, ax, ay * ay)) - c0.z);
      ax = px - c1.x, ay = py - c1.y;
      d1 = fminf(d1, fast_sqrt(fmaf(ax, ax, ay * ay)) - c1.z);
    }
    if (j < e.n_obs) {
      const float4 c = o4[j];
      const float ax = px - c.x, ay = py - c.y;
      d0 = fminf(d0, fast_sqrt(fmaf(ax, ax, ay * ay)) - c.z);
    }
    float d = fminf(d0, d1);
    for (int o = 1; o < lanes; o <<= 1) d = fminf(d, __shfl_xor_sync(0xffffffffu, d, o));
    return d;
  }

  // Nearest cylinder surface: over the candidate list of the point's grid cell when there is
  // a grid and the point is inside it, else over every cylinder (the same float either way).
  // The first kNearestWindow entries of a list are read as one unrolled window whose
  // positions past the list's end repeat its last entry (a repeat leaves a minimum unchanged),
  // so their loads are independent and issue together; longer lists finish in a loop.
  static constexpr int kNearestWindow = 8;
  __device__ __forceinline__ static float nearest(const Env &e, float px, float py) {
    const float gx = (px - e.grid_ox) * e.grid_inv_h, gy = (py - e.grid_oy) * e.grid_inv_h;
    if (e.grid_nx > 0 && gx >= 0.0f && gy >= 0.0f && gx < static_cast<float>(e.grid_nx) &&
        gy < static_cast<float>(e.grid_ny)) {
      const int cell = static_cast<int>(gy) * e.grid_nx + static_cast<int>(gx);
      const float4 *o4 = reinterpret_cast<const float4 *>(e.obs);
      const int t0 = e.grid_off[cell], t1 = e.grid_off[cell + 1];  // t1 > t0: every list holds one
      float dw[kNearestWindow];
#pragma unroll
      for (int q = 0; q < kNearestWindow; ++q) {
        const float4 c = o4[e.grid_idx[min(t0 + q, t1 - 1)]];
        const float ax = px - c.x, ay = py - c.y;
        dw[q] = fast_sqrt(fmaf(ax, ax, ay * ay)) - c.z;
      }
#pragma unroll
      for (int w = kNearestWindow / 2; w > 0; w >>= 1)
#pragma unroll
        for (int q = 0; q < w; ++q) dw[q] = fminf(dw[q], dw[q + w]);
      float d = dw[0];
      for (int t = t0 + kNearestWindow; t < t1; ++t) {
        const float4 c = o4[e.grid_idx[t]];
        const float ax = px - c.x, ay = py - c.y;
        d = fminf(d, fast_sqrt(fmaf(ax, ax, ay * ay)) - c.z);
      }
      return d;
    }
    return obstacle_distance(e, px, py);
  }

  __device__ __forceinline__ static void init(const float *x, Aux &a, const Env &e) {
    a.crashed = false;
    a.d = nearest(e, x[0], x[1]);
  }

  __device__ __forceinline__ static void deriv(const float x[N], const float f[M], float d[N]) {
    const float F = f[0] + f[1] + f[2] + f[3];
    const float tx = arm * (f[1] - f[3]);
    const float ty = arm * (f[2] - f[0]);
    const float tz = kappa * (f[0] - f[1] + f[2] - f[3]);
    float sph, cph, sth, cth, sps, cps;
    __sincosf(x[6], &sph, &cph);
    __sincosf(x[7], &sth, &cth);
    __sincosf(x[8], &sps, &cps);
    const float a = F * (1.0f / mass);
    d[0] = x[3];
    d[1] = x[4];
    d[2] = x[5];
    d[3] = a * (cps * sth * cph + sps * sph);
    d[4] = a * (sps * sth * cph - cps * sph);
    d[5] = a * (cth * cph) - g;
    const float wp = x[9], wq = x[10], wr = x[11];
    const float ws = wq * sph + wr * cph;
    const float inv_cth = __fdividef(1.0f, cth);
    d[6] = wp + ws * sth * inv_cth;
    d[7] = wq * cph - wr * sph;
    d[8] = ws * inv_cth;
    d[9] = (tx - (Izz - Iyy) * wq * wr) * (1.0f / Ixx);
    d[10] = (ty - (Ixx - Izz) * wr * wp) * (1.0f / Iyy);
    d[11] = (tz - (Iyy - Ixx) * wp * wq) * (1.0f / Izz);
  }

  // One classical RK4 step y = x + dt/6 (k1 + 2 k2 + 2 k3 + k4); returns whether every
  // component of y is finite.  The stage sums run two state components per packed FP32
  // instruction (each half rounds as the scalar fmaf / + would).
  __device__ __forceinline__ static void stage(const float x[N], float h, const float k[N], float y[N]) {
    const float2 hh = make_float2(h, h);
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const float2 s = fma2(hh, make_float2(k[i], k[i + 1]), make_float2(x[i], x[i + 1]));
      y[i] = s.x;
      y[i + 1] = s.y;
    }
  }
  __device__ __forceinline__ static bool rk4(const float x[N], const float f[M], float dt, float y[N]) {
    float k1[N], k2[N], k3[N], k4[N];
    deriv(x, f, k1);
    stage(x, 0.5f * dt, k1, y);
    deriv(y, f, k2);
    stage(x, 0.5f * dt, k2, y);
    deriv(y, f, k3);
    stage(x, dt, k3, y);
    deriv(y, f, k4);
    bool finite = true;
    const float2 two = make_float2(2.0f, 2.0f), h6 = make_float2(dt / 6.0f, dt / 6.0f);
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      float2 s = fma2(two, make_float2(k2[i], k2[i + 1]), make_float2(k1[i], k1[i + 1]));
      s = fma2(two, make_float2(k3[i], k3[i + 1]), s);
      s = add2(s, make_float2(k4[i], k4[i + 1]));
      s = fma2(h6, s, make_float2(x[i], x[i + 1]));
      y[i] = s.x;
      y[i + 1] = s.y;
      finite = finite && isfinite(s.x) && isfinite(s.y);
    }
    return finite;
  }

  __device__ __forceinline__ static void step(float x[N], const float f[M], Aux &a, const Env &e, float dt) {
    if (a.crashed) return;
    float y[N];
    const bool finite = rk4(x, f, dt, y);
    const float d = finite ? nearest(e, y[0], y[1]) : -1.0f;
    const bool hit = !finite || d < 0.0f || y[2] < 0.0f || (pitch_limit - fabsf(y[7])) <= 0.0f;
    if (hit) {
      a.crashed = true;  // state stays at the last valid state
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = y[i];
      a.d = d;
    }
  }

  // step() for a lane group holding one sample: the RK4 step is taken by every lane (and by
  // crashed samples, whose result is then discarded) so that the lanes of a warp stay together
  // through the shuffles of the obstacle distance.  Same result as step().
  __device__ __forceinline__ static void step_lanes(float x[N], const float f[M], Aux &a, const Env &e, float dt,
                                                    int sub, int lanes) {
    float y[N];
    const bool finite = rk4(x, f, dt, y);
    float d = obstacle_distance_lanes(e, y[0], y[1], sub, lanes);
    if (!finite) d = -1.0f;
    const bool hit = !finite || d < 0.0f || y[2] < 0.0f || (pitch_limit - fabsf(y[7])) <= 0.0f;
    if (!a.crashed && !hit) {
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] = y[i];
      a.d = d;
    }
    a.crashed = a.crashed || hit;
  }

  __device__ __forceinline__ static float cost(const float x[N], const Aux &a, const Env &e) {
    const float ex = x[0] - e.gx, ey = x[1] - e.gy, ez = x[2] - e.gz;
    float c = w_xy * ex * ex + w_xy * ey * ey + w_z * ez * ez + w_yaw * x[8] * x[8] +
              w_v * (x[3] * x[3] + x[4] * x[4] + x[5] * x[5]) + w_obs * __expf(-a.d * (1.0f / obs_scale));
    return a.crashed ? c + w_crash : c;
  }

  struct Pending {
    float q;
  };
  __device__ __forceinline__ static Pending cost_issue(const float x[N], const Aux &a, const Env &e) {
    return Pending{cost(x, a, e)};
  }
  __device__ __forceinline__ static float cost_finish(const Pending &pd, const Env &) { return pd.q; }
};

}  // namespace mppi

// legged.cu -- Alg. 2 batch rollout and cost for a floating-base planar chain
// with spring-damper ground contact (the legged task model).
//
// Generalised coordinates on the GPU are the base point p = (x, y) (the
// proximal end of link 0) and the absolute link angles phi_j.  For uniform
// thin rods the Lagrangian is
//   T = m |p'|^2 / 2 + p' . sum_j lb_j w_j e'_j + sum_jk D_jk cos(phi_j - phi_k) w_j w_k / 2,
// with lb_j = l_j (m_j/2 + sum_{i>j} m_i), e'_j = (-sin phi_j, cos phi_j) and
// D_jk as for the fixed-base chain.  Eliminating p'' (Schur complement)
// leaves the SPD system
//   sum_k (D_jk - lb_j lb_k / m) cos(phi_j - phi_k) phi''_k = R_j - lb_j e'_j . R_p / m,
// which keeps the cos(phi_j - phi_k) structure, so the same unrolled
// register Cholesky applies; p'' = (R_p - sum_j lb_j e'_j phi''_j) / m.
// Contact forces at the 17 link end points enter through suffix sums (a
// force at the distal end of link c acts on every phi_j with j <= c), the
// velocity terms through the O(L) prefix / suffix form.  Per-thread vectors
// (angles, velocities, sines, cosines, per-sample constants) are staged in
// shared memory so the 16 x 16 factor fits the register file.
#include "rollout_common.cuh"

namespace mtp {
namespace {

constexpr int kLegThreads = 64;

// tanh(x) = 1 - 2 / (exp(2x) + 1) with the SFU exponential and an
// approximate division: the smoothed Coulomb friction direction.  Exact at
// both limits (exp overflows to inf, or underflows to 0); absolute error
// about 1e-7 elsewhere, which scales a friction force of at most mu * fn.
__device__ __forceinline__ float smooth_sign(float x) {
  return 1.f - __fdividef(2.f, __expf(2.f * x) + 1.f);
}

template <int NL>
__device__ __forceinline__ void rollout_legged_body(const RolloutArgs& a, const LeggedModel& lm,
                                                    int r, float* my) {
  constexpr int NC = NL - 1;   // joint torques
  constexpr int NQ = NL + 2;   // generalised coordinates of the state
  constexpr int BD = kLegThreads;
  // thread-private shared-memory vectors, thread-minor (conflict free)
  float* PHI = my;
  float* OMG = my + NL * BD;
  float* CS = my + 2 * NL * BD;
  float* SN = my + 3 * NL * BD;
  float* LB = my + 4 * NL * BD;
  float* WV = my + 5 * NL * BD;
  float* SD = my + 6 * NL * BD;
  float* SA = my + 7 * NL * BD;  // velocity-term suffix sums
  float* SB = my + 8 * NL * BD;
  float* TN = my + 9 * NL * BD;  // torques of steps t and t + 1 (two slots of NC)

  const int b = a.row0 + r;
  const uint32_t iter = a.d_iter ? *a.d_iter : a.iter;
  const float* Ub = a.U + (size_t)r * a.H * NC;
  const int models = (a.dr_mode == MTP_DR_SHARED) ? a.R : 1;
  const float dt = a.dt;
  float total = 0.f;
  for (int mdl = 0; mdl < models; ++mdl) {
    const uint32_t unit = (a.dr_mode == MTP_DR_SHARED) ? (uint32_t)mdl : (uint32_t)b;
    float scl[NL + 1];
    dr_scales<NL + 1>(a, iter, unit, scl);
    const float mu_s = lm.mu_friction * scl[NL];
    float m_tot;
    {
      float outer = 0.f;
#pragma unroll
      for (int j = NL - 1; j >= 0; --j) {
        const float mj = lm.mass[j] * scl[j];
        const float l = lm.length[j];
        LB[j * BD] = l * fmaf(0.5f, mj, outer);
        SD[j * BD] = l * l * fmaf(mj, 1.f / 3.f, outer);
        outer += mj;
      }
      m_tot = outer;
    }
    const float invm = 1.f / m_tot;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const float lb = LB[j * BD];
      WV[j * BD] = fmaf(-lb, invm, lm.length[j]);       // l_j - lb_j / m
      SD[j * BD] = fmaf(-lb * lb, invm, SD[j * BD]);    // D_jj - lb_j^2 / m
    }
    float px = a.x0[0], py = a.x0[1], vx = a.x0[NQ], vy = a.x0[NQ + 1];
    {
      float ph = 0.f, om = 0.f;
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        ph += a.x0[2 + j];
        om += a.x0[NQ + 2 + j];
        PHI[j * BD] = ph;
        OMG[j * BD] = om;
      }
    }
    if (a.X) {
      for (int k = 0; k < 2 * NQ; ++k) a.X[k] = a.x0[k];
    }
    KahanSum J;
    // the torques of step t + 1 are copied into shared memory asynchronously
    // while step t is computed (a plain load stored to shared memory would
    // stall at the store until the load returned)
#pragma unroll
    for (int j = 0; j < NC; ++j) copy_async_f32(TN + j * BD, Ub + j);
    copy_async_commit();
    for (int t = 0; t < a.H; ++t) {
      float* slot = TN + (t & 1) * NC * BD;
      copy_async_wait_all();  // step t's torques (issued one step ago)
      if (t + 1 < a.H) {
        float* next = TN + ((t + 1) & 1) * NC * BD;
#pragma unroll
        for (int j = 0; j < NC; ++j) copy_async_f32(next + j * BD, Ub + (size_t)(t + 1) * NC + j);
        copy_async_commit();
      }
      float tau[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) tau[j] = slot[j * BD];
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        float sj, cj;
        sincos_reduced(PHI[j * BD], &sj, &cj);
        SN[j * BD] = sj;
        CS[j * BD] = cj;
      }
      // stage cost c(x_t, u_t): height, pitch and forward velocity of the
      // base link plus the torque penalty
      {
        float tt = 0.f;
#pragma unroll
        for (int j = 0; j < NC; ++j) tt = fmaf(tau[j], tau[j], tt);
        const float dh = py - lm.target[0], dv = vx - lm.target[1], dp = PHI[0] - lm.target[2];
        const float state = fmaf(lm.w_height, dh * dh, fmaf(lm.w_pitch, dp * dp, lm.w_vel * dv * dv));
        J.add_branch_free(fmaf(lm.w_ctrl, tt, state), a.kahan);
      }
      // generalised forces of the torques and gravity on the link angles
      float rhs[NL];
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        const float tj = (j >= 1) ? tau[j - 1] : 0.f;
        const float tj1 = (j + 1 <= NC) ? tau[j] : 0.f;
        rhs[j] = fmaf(-lm.gravity * LB[j * BD], CS[j * BD], tj - tj1);
      }
      // contact: walk from the tip back to the base, accumulating the force
      // sum over the points beyond each link
      float cx = px, cy = py, cvx = vx, cvy = vy;
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        const float l = lm.length[j], w = OMG[j * BD];
        cx = fmaf(l, CS[j * BD], cx);
        cy = fmaf(l, SN[j * BD], cy);
        cvx = fmaf(-l * w, SN[j * BD], cvx);
        cvy = fmaf(l * w, CS[j * BD], cvy);
      }
      float Fx = 0.f, Fy = 0.f;
#pragma unroll
      for (int c = NL; c >= 0; --c) {
        // branch-free: a point above the ground gets a zero normal force (a
        // divergent branch per point cost more than the arithmetic it skipped)
        const float fn_in = fmaxf(fmaf(-lm.k_contact, cy, -lm.c_contact * cvy), 0.f);
        const float fn = cy < 0.f ? fn_in : 0.f;
        Fx = fmaf(-mu_s * fn, smooth_sign(cvx * lm.inv_v_slip), Fx);
        Fy += fn;
        if (c >= 1) {
          const int j = c - 1;
          const float l = lm.length[j], w = OMG[j * BD];
          const float sj = SN[j * BD], cj = CS[j * BD];
          rhs[j] = fmaf(l, fmaf(-sj, Fx, cj * Fy), rhs[j]);
          cx = fmaf(-l, cj, cx);
          cy = fmaf(-l, sj, cy);
          cvx = fmaf(l * w, sj, cvx);
          cvy = fmaf(-l * w, cj, cvy);
        }
      }
      // velocity terms sum_k D_jk sin(phi_j - phi_k) w_k^2 (prefix / suffix
      // sums), and the base equation's right-hand side
      float Rx = Fx, Ry = fmaf(-m_tot, lm.gravity, Fy);
      {
        float Sa = 0.f, Sb = 0.f;
#pragma unroll
        for (int k = NL - 1; k >= 0; --k) {
          SA[k * BD] = Sa;
          SB[k * BD] = Sb;
          const float w2 = OMG[k * BD] * OMG[k * BD];
          Sa = fmaf(LB[k * BD], CS[k * BD] * w2, Sa);
          Sb = fmaf(LB[k * BD], SN[k * BD] * w2, Sb);
        }
        Rx += Sa;  // sum_j lb_j cos(phi_j) w_j^2
        Ry += Sb;  // sum_j lb_j sin(phi_j) w_j^2
        float Pa = 0.f, Pb = 0.f;
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const float l = lm.length[j], lb = LB[j * BD];
          const float sj = SN[j * BD], cj = CS[j * BD];
          const float ca = fmaf(lb, Pa, l * SA[j * BD]);
          const float cb = fmaf(lb, Pb, l * SB[j * BD]);
          rhs[j] = rhs[j] - fmaf(sj, ca, -cj * cb);
          const float w2 = OMG[j * BD] * OMG[j * BD];
          Pa = fmaf(l, cj * w2, Pa);
          Pb = fmaf(l, sj * w2, Pb);
        }
      }
      // Schur right-hand side
#pragma unroll
      for (int j = 0; j < NL; ++j)
        rhs[j] = fmaf(-LB[j * BD] * invm, fmaf(-SN[j * BD], Rx, CS[j * BD] * Ry), rhs[j]);
      // Schur system S phi'' = rhs.  Below the diagonal S_jk = u_j . v_k with
      // u_j = lb_j (cos phi_j, sin phi_j) and v_k = WV_k (cos phi_k, sin phi_k):
      // a rank-2 semiseparable matrix plus its diagonal SD.  Its Cholesky
      // factor has the same form, L_jk = u_j . w_k below the diagonal, built
      // link by link with the running 2 x 2 matrix M = sum_{i<k} w_i w_i^T:
      //   d_k^2 = SD_k - u_k^T M u_k,  w_k = (v_k - M u_k) / d_k,  M += w_k w_k^T.
      // Then L y = rhs and L^T phi'' = y with running 2-vectors: O(NL) in
      // all, against O(NL^3) for the dense factorisation of the same matrix.
      float u1[NL], u2[NL], w1[NL], w2[NL], dinv[NL];
      {
        float m11 = 0.f, m12 = 0.f, m22 = 0.f;
#pragma unroll
        for (int k = 0; k < NL; ++k) {
          const float ck = CS[k * BD], sk = SN[k * BD], lbk = LB[k * BD], wvk = WV[k * BD];
          u1[k] = lbk * ck;
          u2[k] = lbk * sk;
          const float mu1 = fmaf(m11, u1[k], m12 * u2[k]);
          const float mu2 = fmaf(m12, u1[k], m22 * u2[k]);
          const float inv = rsqrtf(SD[k * BD] - fmaf(u1[k], mu1, u2[k] * mu2));
          dinv[k] = inv;
          w1[k] = fmaf(wvk, ck, -mu1) * inv;
          w2[k] = fmaf(wvk, sk, -mu2) * inv;
          m11 = fmaf(w1[k], w1[k], m11);
          m12 = fmaf(w1[k], w2[k], m12);
          m22 = fmaf(w2[k], w2[k], m22);
        }
      }
      {
        float z1 = 0.f, z2 = 0.f;
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          rhs[j] = (rhs[j] - fmaf(u1[j], z1, u2[j] * z2)) * dinv[j];
          z1 = fmaf(w1[j], rhs[j], z1);
          z2 = fmaf(w2[j], rhs[j], z2);
        }
        float r1 = 0.f, r2 = 0.f;
#pragma unroll
        for (int k = NL - 1; k >= 0; --k) {
          rhs[k] = (rhs[k] - fmaf(w1[k], r1, w2[k] * r2)) * dinv[k];
          r1 = fmaf(u1[k], rhs[k], r1);
          r2 = fmaf(u2[k], rhs[k], r2);
        }
      }
      // base acceleration, then semi-implicit Euler
      float ax = Rx, ay = Ry;
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        const float g = LB[j * BD] * rhs[j];
        ax = fmaf(g, SN[j * BD], ax);   // - lb_j (-sin phi_j) phi''_j
        ay = fmaf(-g, CS[j * BD], ay);  // - lb_j cos(phi_j) phi''_j
      }
      vx = fmaf(dt, ax * invm, vx);
      vy = fmaf(dt, ay * invm, vy);
      px = fmaf(dt, vx, px);
      py = fmaf(dt, vy, py);
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        const float w = fmaf(dt, rhs[j], OMG[j * BD]);
        OMG[j * BD] = w;
        PHI[j * BD] = fmaf(dt, w, PHI[j * BD]);
      }
      if (a.X) {
        float* xo = a.X + (size_t)(t + 1) * 2 * NQ;
        xo[0] = px;
        xo[1] = py;
        xo[NQ] = vx;
        xo[NQ + 1] = vy;
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          xo[2 + j] = PHI[j * BD] - (j ? PHI[(j - 1) * BD] : 0.f);
          xo[NQ + 2 + j] = OMG[j * BD] - (j ? OMG[(j - 1) * BD] : 0.f);
        }
      }
    }
    {
      const float dh = py - lm.target[0], dv = vx - lm.target[1], dp = PHI[0] - lm.target[2];
      const float state = fmaf(lm.w_height, dh * dh, fmaf(lm.w_pitch, dp * dp, lm.w_vel * dv * dv));
      J.add_branch_free(lm.w_term * state, a.kahan);
    }
    total += J.s;
  }
  float cst = total / (float)models;
  if (!isfinite(cst)) cst = __int_as_float(0x7f800000);
  a.cost[r] = cst;
}

template <int NL>
__global__ void __launch_bounds__(kLegThreads) k_rollout_legged(const RolloutArgs a,
                                                                const LeggedModel lm) {
  __shared__ float sh[(9 * NL + 2 * (NL - 1)) * kLegThreads];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.rows) return;
  rollout_legged_body<NL>(a, lm, r, sh + threadIdx.x);
}

template <int NL>
__global__ void __launch_bounds__(kLegThreads) k_rollout_legged_batch(
    const RolloutArgs* __restrict__ ra, const LeggedModel* __restrict__ lms,
    const int* __restrict__ row_start, int count) {
  __shared__ float sh[(9 * NL + 2 * (NL - 1)) * kLegThreads];
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= __ldg(row_start + count)) return;
  const int i = batch_instance(row_start, count, g);
  const RolloutArgs a = ra[i];
  const int r = g - __ldg(row_start + i);
  if (r >= a.rows) return;
  rollout_legged_body<NL>(a, lms[i], r, sh + threadIdx.x);
}

template <int NL>
cudaError_t legged_dispatch(const RolloutArgs& a, const LeggedModel& m, int links, cudaStream_t s) {
  if constexpr (NL <= 16) {
    if (links == NL) {
      k_rollout_legged<NL><<<(a.rows + kLegThreads - 1) / kLegThreads, kLegThreads, 0, s>>>(a, m);
      return cudaGetLastError();
    }
    return legged_dispatch<NL + 1>(a, m, links, s);
  } else {
    return cudaErrorInvalidValue;
  }
}

template <int NL>
cudaError_t legged_batch_dispatch(const RolloutArgs* ra, const LeggedModel* lm, const int* rs,
                                  int count, int total_rows, int links, cudaStream_t s) {
  if constexpr (NL <= 16) {
    if (links == NL) {
      k_rollout_legged_batch<NL><<<(total_rows + kLegThreads - 1) / kLegThreads, kLegThreads, 0, s>>>(
          ra, lm, rs, count);
      return cudaGetLastError();
    }
    return legged_batch_dispatch<NL + 1>(ra, lm, rs, count, total_rows, links, s);
  } else {
    return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_rollout_legged(const RolloutArgs& a, const LeggedModel& m, int links,
                                  cudaStream_t s) {
  if (a.rows <= 0) return cudaSuccess;
  return legged_dispatch<2>(a, m, links, s);
}

cudaError_t launch_rollout_legged_batch(const RolloutArgs* d_ra, const LeggedModel* d_lm,
                                        const int* d_row_start, int count, int total_rows,
                                        int links, cudaStream_t s) {
  if (total_rows <= 0) return cudaSuccess;
  return legged_batch_dispatch<2>(d_ra, d_lm, d_row_start, count, total_rows, links, s);
}

}  // namespace mtp

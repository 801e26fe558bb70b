// rollout_kernels.cuh -- Alg. 2 batch rollout fused with the cost reduction
// (Eq. 2) for the k-D point mass and the planar serial chain: the device
// bodies and kernels, instantiated by rollout_pm.cu and rollout_chain.cu.
//
// One thread per candidate keeps the whole state in registers for all H
// steps and accumulates c(x_t, u_t) with compensated FP32 sums; only the
// final cost leaves the SM.  The loop bodies are fully unrolled over the
// compile-time dimension (point-mass axes, chain links), so the per-step
// linear algebra lives in registers.  The controls reach a thread either by
// direct loads a few steps ahead (T = 0) or staged through shared memory a
// horizon chunk of T steps at a time by bulk copies (T = 4, 8; see
// StagedRows): the chunk length is the rollout tile's horizon chunk, picked
// per launch shape by the batch autotuner.
//
// Planar chain: the dynamics are evaluated in absolute link angles phi_j
// (phi_j = q_1 + ... + q_j).  For uniform thin rods the Lagrangian gives the
// mass matrix A_jk = D_jk cos(phi_j - phi_k) with constant D (from the link
// masses and lengths), velocity terms D_jk sin(phi_j - phi_k) w_k^2, gravity
// g l_j beta_j cos(phi_j) and generalised forces tau_j - tau_{j+1}; the
// SPD system is solved by an unrolled Cholesky.  Semi-implicit Euler in
// (phi, w) equals semi-implicit Euler in the relative joint coordinates.
#pragma once

#include "rollout_common.cuh"

namespace mtp {
namespace {

constexpr int kThreads = 128;
// Chains of at least this many links solve their mass matrix by the O(NL)
// semiseparable Cholesky, shorter ones by the dense factor.  At 7 links the
// dense factor is the faster of the two: as fast in a batch, and 99 -> 79 us
// for a lone 4096-candidate arm, whose one warp per SM sub-partition runs
// the step's serial chain (the recursion's is longer).
#ifndef MTP_SEMISEP_LINKS
#define MTP_SEMISEP_LINKS 8
#endif
constexpr int kSemisepLinks = MTP_SEMISEP_LINKS;

// Threads per block: fill as many SMs as the batch allows (one thread per
// candidate; small batches get one warp per block).
inline int rollout_block(int rows) {
  const int sms = device_sms();
  int bd = 128;
  while (bd > 32 && (rows + bd - 1) / bd < sms) bd >>= 1;
  return bd;
}

// Dynamic shared memory of a rollout block of `block` threads staging K
// controls per step T steps at a time (0 for direct loads).
template <int K, int T>
constexpr size_t staged_smem(int block) {
  if constexpr (T == 0) return 0;
  else return (size_t)(block / 32) * StageShape<K, T>::kWarpBytes;
}

// This warp's staging area in the block's dynamic shared memory.
__device__ __forceinline__ unsigned char* warp_stage_area(size_t warp_bytes) {
  extern __shared__ __align__(16) unsigned char rollout_dyn_smem[];
  return rollout_dyn_smem + (threadIdx.x >> 5) * warp_bytes;
}

__device__ __forceinline__ void report_stage_timeout(const RolloutArgs& a) {
  if (a.status) atomicOr(a.status, kStatusStageTimeout);
}

// ---------------------------------------------------------------------------
// k-D point mass (double integrator), control = acceleration x gain.
// ---------------------------------------------------------------------------
// ALL: every obstacle slot is evaluated, with no branch (the slots past
// n_obs have radius 0 and add exactly +0): one basic block, so the obstacles'
// SFU latencies overlap, for a lone latency-bound instance (measured on the
// C1 point mass: rollout 26.0 -> 20.5 us).  Otherwise the slots past n_obs
// are skipped, which saves their instructions where many instances keep the
// GPU busy (the batch of 256: 3.84 -> 3.72 ms).  The sums are the same bits.
template <int K, bool ALL>
__device__ __forceinline__ float pm_state_cost(const PointMassModel& pm, const float (&p)[K]) {
  float dist2 = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float e = p[k] - pm.target[k];
    dist2 = fmaf(e, e, dist2);
  }
  // unrolled to the maximum obstacle count so every model index is a
  // constant (a run-time index into the kernel parameters goes through the
  // constant cache's slow indexed path)
  float pen = 0.f;
#pragma unroll
  for (int o = 0; o < MTP_MAX_OBSTACLES; ++o) {
    if (ALL || o < pm.n_obs) {
      float d2 = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float e = p[k] - pm.obs_c[o][k];
        d2 = fmaf(e, e, d2);
      }
      // distance as d2 * rsqrt(d2): one SFU operation and a multiply instead
      // of the correctly rounded square root's fix-up sequence (relative
      // error ~1e-7, far inside the cost tolerance)
      const float dist = d2 > 0.f ? d2 * rsqrtf(d2) : 0.f;
      const float depth = pm.obs_r[o] - dist;
      pen += depth > 0.f ? depth : 0.f;
    }
  }
  return fmaf(pm.w_target, dist2, pm.w_obs * pen);
}

// The K controls of step t drive v += dt g u, p += dt v (g: the per-model
// control gains of the domain randomisation); the stage cost is taken
// before the step and the terminal cost on the final state.
template <int K, int PF, bool ALL, int T>
__device__ __forceinline__ bool rollout_pm_body(const RolloutArgs& a, const PointMassModel& pm,
                                                int r, bool live, StagedRows<K, T>* st) {
  const int b = a.row0 + r;
  const uint32_t iter = a.d_iter ? *a.d_iter : a.iter;
  const float* Ub = a.U + (size_t)r * a.H * K;
  const int models = (a.dr_mode == MTP_DR_SHARED) ? a.R : 1;
  const float dt = a.dt;
  float total = 0.f;
  bool ok = true;
  for (int mdl = 0; mdl < models && ok; ++mdl) {
    const uint32_t unit = (a.dr_mode == MTP_DR_SHARED) ? (uint32_t)mdl : (uint32_t)b;
    float gain[K], p[K], v[K];
    dr_scales<K>(a, iter, unit, gain);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      gain[k] *= dt;
      p[k] = a.x0[k];
      v[k] = a.x0[K + k];
    }
    if (a.X) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        a.X[k] = p[k];
        a.X[K + k] = v[k];
      }
    }
    KahanSum J;
    ok = for_each_step<K, PF, T>(Ub, a.H, st, [&](int t, const float (&u)[K]) {
      float uu = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) uu = fmaf(u[k], u[k], uu);
      J.add(fmaf(pm.w_ctrl, uu, pm_state_cost<K, ALL>(pm, p)), a.kahan);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        v[k] = fmaf(gain[k], u[k], v[k]);
        p[k] = fmaf(dt, v[k], p[k]);
      }
      if (a.X) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
          a.X[(size_t)(t + 1) * 2 * K + k] = p[k];
          a.X[(size_t)(t + 1) * 2 * K + K + k] = v[k];
        }
      }
    });
    J.add(pm.w_term * pm_state_cost<K, ALL>(pm, p), a.kahan);
    total += J.s;
  }
  if (!live) return ok;
  float c = total / (float)models;
  if (!isfinite(c) || !ok) c = __int_as_float(0x7f800000);
  if (!ok) report_stage_timeout(a);
  a.cost[r] = c;
  return ok;
}

// ---------------------------------------------------------------------------
// Planar serial chain under joint torques.
// ---------------------------------------------------------------------------
// Two candidates per thread (rows r[0] and r[1] of one instance, 32 rows
// apart), direct loads one step ahead, one model: the two chains of
// dependent instructions interleave, which the point-mass step needs (its
// warps otherwise stall on fixed-latency dependencies most of the time).
// Same arithmetic per candidate as rollout_pm_body, so the same bits.  A
// candidate without a row (live false) reads the instance's first row and
// writes nothing.  One model per candidate (no shared-model averaging).
template <int K>
__device__ __forceinline__ void rollout_pm_pair(const RolloutArgs& a, const PointMassModel& pm,
                                                const int (&r)[2], const bool (&live)[2]) {
  constexpr int S = 2;
  const uint32_t iter = a.d_iter ? *a.d_iter : a.iter;
  const float dt = a.dt;
  const int H = a.H;
  const float* Ub[S];
  float gain[S][K], p[S][K], v[S][K];
  KahanSum J[S];
#pragma unroll
  for (int c = 0; c < S; ++c) {
    Ub[c] = a.U + (size_t)(live[c] ? r[c] : 0) * H * K;
    dr_scales<K>(a, iter, (uint32_t)(a.row0 + r[c]), gain[c]);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      gain[c][k] *= dt;
      p[c][k] = a.x0[k];
      v[c][k] = a.x0[K + k];
    }
  }
  float ub[S][K];
#pragma unroll
  for (int c = 0; c < S; ++c)
#pragma unroll
    for (int k = 0; k < K; ++k) ub[c][k] = __ldg(Ub[c] + k);
  for (int t = 0; t < H; ++t) {
    const int tn = min(t + 1, H - 1);
#pragma unroll
    for (int c = 0; c < S; ++c) {
      float u[K];
      float uu = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        u[k] = ub[c][k];
        ub[c][k] = __ldg(Ub[c] + tn * K + k);
        uu = fmaf(u[k], u[k], uu);
      }
      J[c].add(fmaf(pm.w_ctrl, uu, pm_state_cost<K, false>(pm, p[c])), a.kahan);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        v[c][k] = fmaf(gain[c][k], u[k], v[c][k]);
        p[c][k] = fmaf(dt, v[c][k], p[c][k]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < S; ++c) {
    J[c].add(pm.w_term * pm_state_cost<K, false>(pm, p[c]), a.kahan);
    if (live[c]) {
      float cst = J[c].s;
      if (!isfinite(cst)) cst = __int_as_float(0x7f800000);
      a.cost[r[c]] = cst;
    }
  }
}

template <int NL>
__device__ __forceinline__ void chain_tip(const float (&len)[NL], const float (&c)[NL],
                                          const float (&s)[NL], float& x, float& y) {
  x = 0.f;
  y = 0.f;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    x = fmaf(len[j], c[j], x);
    y = fmaf(len[j], s[j], y);
  }
}

template <int NL, int PF, int T>
__device__ __forceinline__ bool rollout_chain_body(const RolloutArgs& a, const ChainModel& cm,
                                                   int r, bool live, StagedRows<NL, T>* st) {
  const int b = a.row0 + r;
  const uint32_t iter = a.d_iter ? *a.d_iter : a.iter;
  const float* Ub = a.U + (size_t)r * a.H * NL;
  const int models = (a.dr_mode == MTP_DR_SHARED) ? a.R : 1;
  const float dt = a.dt;
  float len[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) len[j] = cm.length[j];
  float total = 0.f;
  bool ok = true;
  for (int mdl = 0; mdl < models && ok; ++mdl) {
    const uint32_t unit = (a.dr_mode == MTP_DR_SHARED) ? (uint32_t)mdl : (uint32_t)b;
    // Lagrangian constants: beta_j = m_j/2 + sum_{i>j} m_i, lb_j = l_j beta_j,
    // D_jj = l_j^2 (m_j/3 + sum_{i>j} m_i), G_j = g l_j beta_j.
    float lb[NL], Dd[NL], G[NL];
    {
      float mass[NL];
      dr_scales<NL>(a, iter, unit, mass);
#pragma unroll
      for (int j = 0; j < NL; ++j) mass[j] *= cm.mass[j];
      float outer = 0.f;
#pragma unroll
      for (int j = NL - 1; j >= 0; --j) {
        const float beta = fmaf(0.5f, mass[j], outer);
        lb[j] = len[j] * beta;
        Dd[j] = len[j] * len[j] * fmaf(mass[j], 1.f / 3.f, outer);
        G[j] = cm.gravity * lb[j];
        outer += mass[j];
      }
    }
    float phi[NL], w[NL];
    {
      float ph = 0.f, om = 0.f;
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        ph += a.x0[j];
        om += a.x0[NL + j];
        phi[j] = ph;
        w[j] = om;
      }
    }
    if (a.X) {
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        a.X[j] = a.x0[j];
        a.X[NL + j] = a.x0[NL + j];
      }
    }
    KahanSum J;
    ok = for_each_step<NL, PF, T>(Ub, a.H, st, [&](int t, const float (&u)[NL]) {
      float c[NL], s[NL], tau[NL];
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        tau[j] = u[j];
        sincos_reduced(phi[j], &s[j], &c[j]);
      }
      // stage cost c(x_t, u_t): reach error of the tip and torque penalty
      {
        float x, y;
        chain_tip<NL>(len, c, s, x, y);
        const float ex = x - cm.target[0], ey = y - cm.target[1];
        float tt = 0.f;
#pragma unroll
        for (int j = 0; j < NL; ++j) tt = fmaf(tau[j], tau[j], tt);
        J.add(fmaf(cm.w_target, fmaf(ex, ex, ey * ey), cm.w_ctrl * tt), a.kahan);
      }
      // right-hand side: generalised forces and gravity
      float rhs[NL];
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        const float q_next = (j + 1 < NL) ? tau[j + 1] : 0.f;
        rhs[j] = fmaf(-G[j], c[j], tau[j] - q_next);
      }
      // the dense mass matrix (lower triangle) of the shorter chains, built
      // before the velocity terms so that its independent products overlap
      // their prefix sums: A_jk = D_jk cos(phi_j - phi_k) with D_jk = l_k lb_j
      // below the diagonal
      using Tr = Tri<NL>;
      float A[Tr::size];
      if constexpr (NL < kSemisepLinks) {
#pragma unroll
        for (int j = 0; j < NL; ++j) A[Tr::at(j, j)] = Dd[j];
        Unroll<1, NL>::run([&](auto J) {
          constexpr int j = decltype(J)::value;
          Unroll<0, j>::run([&](auto K) {
            constexpr int k = decltype(K)::value;
            A[Tr::at(j, k)] = (len[k] * lb[j]) * fmaf(c[j], c[k], s[j] * s[k]);  // cos(phi_j - phi_k)
          });
        });
      }
      // velocity terms sum_k D_jk sin(phi_j - phi_k) w_k^2 in O(NL): with
      // a_k = c_k w_k^2, b_k = s_k w_k^2 the sum is
      // s_j (lb_j Pa_j + l_j Sa_j) - c_j (lb_j Pb_j + l_j Sb_j), where P sums
      // l_k (.)_k over k < j and S sums lb_k (.)_k over k > j
      {
        float wa[NL], wb[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
          const float w2 = w[k] * w[k];
          wa[k] = c[k] * w2;
          wb[k] = s[k] * w2;
        }
        float Pa = 0.f, Pb = 0.f;
        float Sa[NL], Sb[NL];
        Sa[NL - 1] = 0.f;
        Sb[NL - 1] = 0.f;
#pragma unroll
        for (int k = NL - 2; k >= 0; --k) {
          Sa[k] = fmaf(lb[k + 1], wa[k + 1], Sa[k + 1]);
          Sb[k] = fmaf(lb[k + 1], wb[k + 1], Sb[k + 1]);
        }
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          const float ca = fmaf(lb[j], Pa, len[j] * Sa[j]);
          const float cb = fmaf(lb[j], Pb, len[j] * Sb[j]);
          rhs[j] = rhs[j] - fmaf(s[j], ca, -c[j] * cb);
          Pa = fmaf(len[j], wa[j], Pa);
          Pb = fmaf(len[j], wb[j], Pb);
        }
      }
      if constexpr (NL >= kSemisepLinks) {
        // Below the diagonal A_jk = u_j . v_k with u_j = lb_j (cos phi_j,
        // sin phi_j) and v_k = l_k (cos phi_k, sin phi_k): a rank-2
        // semiseparable matrix plus its diagonal Dd.  Its Cholesky factor
        // has the same form, L_jk = u_j . w_k, built link by link with the
        // running 2 x 2 matrix M = sum_{i<k} w_i w_i^T:
        //   d_k^2 = Dd_k - u_k^T M u_k,  w_k = (v_k - M u_k) / d_k,  M += w_k w_k^T;
        // then L y = rhs and L^T phi'' = y with running 2-vectors: O(NL)
        // work and registers, against O(NL^3) work and O(NL^2) registers
        // for the dense factor.
        float u1[NL], u2[NL], w1[NL], w2[NL], dinv[NL];
        float m11 = 0.f, m12 = 0.f, m22 = 0.f;
#pragma unroll
        for (int k = 0; k < NL; ++k) {
          u1[k] = lb[k] * c[k];
          u2[k] = lb[k] * s[k];
          const float mu1 = fmaf(m11, u1[k], m12 * u2[k]);
          const float mu2 = fmaf(m12, u1[k], m22 * u2[k]);
          const float inv = rsqrtf(Dd[k] - fmaf(u1[k], mu1, u2[k] * mu2));
          dinv[k] = inv;
          w1[k] = fmaf(len[k], c[k], -mu1) * inv;
          w2[k] = fmaf(len[k], s[k], -mu2) * inv;
          m11 = fmaf(w1[k], w1[k], m11);
          m12 = fmaf(w1[k], w2[k], m12);
          m22 = fmaf(w2[k], w2[k], m22);
        }
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
      } else {
        float inv[NL];
        // Cholesky A = L L^T in place (inv holds 1 / L_jj), then the two
        // triangular solves
        Unroll<0, NL>::run([&](auto J) {
          constexpr int j = decltype(J)::value;
          float d = A[Tr::at(j, j)];
          Unroll<0, j>::run([&](auto K) {
            constexpr int k = decltype(K)::value;
            d = fmaf(-A[Tr::at(j, k)], A[Tr::at(j, k)], d);
          });
          inv[j] = rsqrtf(d);
          Unroll<j + 1, NL>::run([&](auto I) {
            constexpr int i = decltype(I)::value;
            float v = A[Tr::at(i, j)];
            Unroll<0, j>::run([&](auto K) {
              constexpr int k = decltype(K)::value;
              v = fmaf(-A[Tr::at(i, k)], A[Tr::at(j, k)], v);
            });
            A[Tr::at(i, j)] = v * inv[j];
          });
        });
        Unroll<0, NL>::run([&](auto I) {
          constexpr int i = decltype(I)::value;
          float v = rhs[i];
          Unroll<0, i>::run([&](auto K) {
            constexpr int k = decltype(K)::value;
            v = fmaf(-A[Tr::at(i, k)], rhs[k], v);
          });
          rhs[i] = v * inv[i];
        });
        Unroll<0, NL>::run([&](auto I) {
          constexpr int i = NL - 1 - decltype(I)::value;
          float v = rhs[i];
          Unroll<i + 1, NL>::run([&](auto K) {
            constexpr int k = decltype(K)::value;
            v = fmaf(-A[Tr::at(k, i)], rhs[k], v);
          });
          rhs[i] = v * inv[i];
        });
      }
      // semi-implicit Euler in absolute coordinates
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        w[j] = fmaf(dt, rhs[j], w[j]);
        phi[j] = fmaf(dt, w[j], phi[j]);
      }
      if (a.X) {
        float* xo = a.X + (size_t)(t + 1) * 2 * NL;
#pragma unroll
        for (int j = 0; j < NL; ++j) {
          xo[j] = phi[j] - (j ? phi[j - 1] : 0.f);
          xo[NL + j] = w[j] - (j ? w[j - 1] : 0.f);
        }
      }
    });
    {
      float c[NL], s[NL], x, y;
#pragma unroll
      for (int j = 0; j < NL; ++j) sincos_reduced(phi[j], &s[j], &c[j]);
      chain_tip<NL>(len, c, s, x, y);
      const float ex = x - cm.target[0], ey = y - cm.target[1];
      J.add(cm.w_term * cm.w_target * fmaf(ex, ex, ey * ey), a.kahan);
    }
    total += J.s;
  }
  if (!live) return ok;
  float cst = total / (float)models;
  if (!isfinite(cst) || !ok) cst = __int_as_float(0x7f800000);
  if (!ok) report_stage_timeout(a);
  a.cost[r] = cst;
  return ok;
}

// Standalone launches: one thread per candidate row.  Direct loads (T = 0)
// let threads past the last row leave at once; staged loads keep every lane
// of a warp in the warp's copy protocol.
template <int K, int T>
__global__ void __launch_bounds__(kThreads) k_rollout_pm(const RolloutArgs a,
                                                         const PointMassModel pm) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (T == 0) {
    if (r >= a.rows) return;
    rollout_pm_body<K, kPrefetchAlone, true, 0>(a, pm, r, true, nullptr);
  } else {
    if (__all_sync(0xffffffffu, r >= a.rows)) return;
    const bool live = r < a.rows;
    StagedRows<K, T> st;
    st.init(warp_stage_area(StageShape<K, T>::kWarpBytes), live ? a.U + (size_t)r * a.H * K : nullptr,
            a.H);
    rollout_pm_body<K, kPrefetchAlone, true, T>(a, pm, r, live, &st);
  }
}

// Rows are padded to whole warps, so a warp belongs to one instance: each
// warp copies its instance's model (goal, obstacles) to shared memory once.
// Read from global memory, the obstacle data cost about 6K + 9 loads per
// step through L1; the standalone kernel reads it as constant operands.
template <int K, int T>
__global__ void __launch_bounds__(kThreads) k_rollout_pm_batch(const RolloutArgs* __restrict__ ra,
                                                               const PointMassModel* __restrict__ pm,
                                                               const int* __restrict__ row_start,
                                                               int count) {
  __shared__ PointMassModel models[kThreads / 32];
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= __ldg(row_start + count)) return;  // whole warps: the total is padded to warps
  const int i = batch_instance(row_start, count, g);
  PointMassModel& m = models[threadIdx.x >> 5];
  {
    const int* src = reinterpret_cast<const int*>(pm + i);
    int* dst = reinterpret_cast<int*>(&m);
    for (int w = threadIdx.x & 31; w < (int)(sizeof(PointMassModel) / sizeof(int)); w += 32)
      dst[w] = __ldg(src + w);
    __syncwarp();
  }
  const RolloutArgs a = ra[i];
  const int r = g - __ldg(row_start + i);
  const bool live = r < a.rows;
  if constexpr (T == 0) {
    if (!live) return;
    rollout_pm_body<K, kPrefetchBatch, false, 0>(a, m, r, true, nullptr);
  } else {
    StagedRows<K, T> st;
    st.init(warp_stage_area(StageShape<K, T>::kWarpBytes), live ? a.U + (size_t)r * a.H * K : nullptr,
            a.H);
    rollout_pm_body<K, kPrefetchBatch, false, T>(a, m, r, live, &st);
  }
}

// Batched point masses, two candidates per thread: instances' rows are
// padded to 64, and thread g of the launch takes padded rows 64 (g / 32) +
// (g % 32) and that + 32, which share an instance.
template <int K>
__global__ void __launch_bounds__(kThreads) k_rollout_pm_batch2(const RolloutArgs* __restrict__ ra,
                                                                const PointMassModel* __restrict__ pm,
                                                                const int* __restrict__ row_start,
                                                                int count) {
  __shared__ PointMassModel models[kThreads / 32];
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int r0 = (g >> 5) * 64 + (g & 31);
  if (r0 >= __ldg(row_start + count)) return;  // whole warps: the total is padded to 64
  const int i = batch_instance(row_start, count, r0);
  PointMassModel& m = models[threadIdx.x >> 5];
  {
    const int* src = reinterpret_cast<const int*>(pm + i);
    int* dst = reinterpret_cast<int*>(&m);
    for (int w = threadIdx.x & 31; w < (int)(sizeof(PointMassModel) / sizeof(int)); w += 32)
      dst[w] = __ldg(src + w);
    __syncwarp();
  }
  const RolloutArgs a = ra[i];
  const int r[2] = {r0 - __ldg(row_start + i), r0 - __ldg(row_start + i) + 32};
  const bool live[2] = {r[0] < a.rows, r[1] < a.rows};
  if (!live[0] && !live[1]) return;
  rollout_pm_pair<K>(a, m, r, live);
}

template <int NL, int T>
__global__ void __launch_bounds__(kThreads) k_rollout_chain(const RolloutArgs a,
                                                            const ChainModel cm) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (T == 0) {
    if (r >= a.rows) return;
    rollout_chain_body<NL, kPrefetchAlone, 0>(a, cm, r, true, nullptr);
  } else {
    if (__all_sync(0xffffffffu, r >= a.rows)) return;
    const bool live = r < a.rows;
    StagedRows<NL, T> st;
    st.init(warp_stage_area(StageShape<NL, T>::kWarpBytes),
            live ? a.U + (size_t)r * a.H * NL : nullptr, a.H);
    rollout_chain_body<NL, kPrefetchAlone, T>(a, cm, r, live, &st);
  }
}

template <int NL, int T>
__global__ void __launch_bounds__(kThreads) k_rollout_chain_batch(const RolloutArgs* __restrict__ ra,
                                                                  const ChainModel* __restrict__ cms,
                                                                  const int* __restrict__ row_start,
                                                                  int count) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= __ldg(row_start + count)) return;
  const int i = batch_instance(row_start, count, g);
  const RolloutArgs a = ra[i];
  const ChainModel cm = cms[i];
  const int r = g - __ldg(row_start + i);
  const bool live = r < a.rows;
  if constexpr (T == 0) {
    if (!live) return;
    rollout_chain_body<NL, kPrefetchBatch, 0>(a, cm, r, true, nullptr);
  } else {
    StagedRows<NL, T> st;
    st.init(warp_stage_area(StageShape<NL, T>::kWarpBytes),
            live ? a.U + (size_t)r * a.H * NL : nullptr, a.H);
    rollout_chain_body<NL, kPrefetchBatch, T>(a, cm, r, live, &st);
  }
}

}  // namespace
}  // namespace mtp

// minimize_kernel.cuh -- the persistent FIRE minimiser kernel template (see
// minimize.cu for the design); included by the per-configuration
// instantiation units.
#pragma once
#include <cooperative_groups.h>
#include <math.h>

#include "aqs_internal.cuh"
#include "launch.cuh"
#include "minimize.cuh"

namespace cg = cooperative_groups;

namespace aqs {

// NaN-propagating max for the reductions (a NaN anywhere must reach the
// decision so that every CTA stops together).
__device__ __forceinline__ double nmax(double a, double b) { return (a != a || a > b) ? a : b; }

// Slots 0, 4, 5 are max-reductions, the others sums.
__device__ __forceinline__ bool is_max_slot(int m) { return m == 0 || m == 4 || m == 5; }

template <int D>
__device__ __forceinline__ void pair64(const PairCoef& c, const double* d, double* F, bool want_e,
                                       double& e, double& w) {
  double s = d[0] * d[0];
#pragma unroll
  for (int k = 1; k < D; k++) s = fma(d[k], d[k], s);
  if (s < c.rc2) {
    double u = 1.0 / s;
    double a = rsqrt(s);
    double u3 = u * u * u, u4 = u3 * u, u7 = u4 * u3;
    double phi = fma(c.A, u7, fma(c.B, u4, c.C * a));
#pragma unroll
    for (int k = 0; k < D; k++) F[k] = fma(phi, d[k], F[k]);
    if (want_e) {
      double r = s * a;
      e += c.e12 * u3 * u3 - c.e6 * u3 - c.Uc - (r - c.rc) * c.dUc;
      w = fma(phi * d[0], d[1], w);
    }
  }
}

// FP32 coefficients of one species pair, held in registers by the pair loop
struct Coef32 {
  float Af, Bf, Cf, rc2f;
};
__device__ __forceinline__ Coef32 coef32(const PairCoef& c) { return Coef32{c.Af, c.Bf, c.Cf, c.rc2f}; }

// Force change of one pair between the reference separation d0 and d0 + e,
// in FP32, by divided differences (no cancellation between phi(s) and
// phi(s0)).  With u = 1/s, w = 1/s0, ds = s - s0:
//   (s^-n - s0^-n) / ds = -u w sum_{k<n} u^k w^(n-1-k)
//   (s^-1/2 - s0^-1/2) / ds = -(ab)^2 / (a + b),  a = s^-1/2, b = s0^-1/2
//   dF = phi(s) e + [phi(s) - phi(s0)] d0
// A pair that crosses the cutoff (in the list but inside at only one of the
// two separations) uses the plain difference, with phi = 0 outside.  The
// function has no branches, so the lanes of a warp never diverge on it.
template <int D>
__device__ __forceinline__ void pair_dev(const Coef32& c, const float* d0, const float* e,
                                         float* F) {
  float s0 = d0[0] * d0[0], ds = e[0] * fmaf(2.0f, d0[0], e[0]);
#pragma unroll
  for (int k = 1; k < D; k++) {
    s0 = fmaf(d0[k], d0[k], s0);
    ds = fmaf(e[k], fmaf(2.0f, d0[k], e[k]), ds);
  }
  const float s = s0 + ds;
  const bool in0 = s0 < c.rc2f, in1 = s < c.rc2f;
  const float a = rsqrtf(s), b = rsqrtf(s0);
  const float u = a * a, w = b * b;
  const float w2 = w * w, w3 = w2 * w, w4 = w2 * w2, w5 = w4 * w, w6 = w3 * w3;
  const float h4 = fmaf(u, fmaf(u, w + u, w2), w3);
  const float h7 = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, w + u, w2), w3), w4), w5), w6);
  const float uw = u * w;
  const float ab = a * b;
  const float dh = -__fdividef(ab * ab, a + b);
  const float u2 = u * u, u4 = u2 * u2, u7 = u4 * u2 * u;
  float phi = fmaf(c.Af, u7, fmaf(c.Bf, u4, c.Cf * a));
  const float phi0 = fmaf(c.Af, w4 * w3, fmaf(c.Bf, w4, c.Cf * b));
  const float dd = ds * fmaf(-c.Af * uw, h7, fmaf(-c.Bf * uw, h4, c.Cf * dh));
  phi = in1 ? phi : 0.0f;
  const float dphi = (in0 && in1) ? dd : phi - (in0 ? phi0 : 0.0f);
#pragma unroll
  for (int k = 0; k < D; k++) F[k] += fmaf(phi, e[k], dphi * d0[k]);
}

// Published record of one atom in shared memory.  EVAL64 reads q64 (FP64
// position relative to the atom's cell origin); the mixed FP32 path reads
// (q32, delta32).  The two views alias: each iteration publishes exactly the
// one the next force phase needs, after every CTA has passed the mid-iteration
// barrier.
template <int D>
struct Pub;
template <>
struct Pub<2> {
  union {
    double q64[2];
    float4 p32;  // q.x, q.y, delta.x, delta.y
  };
};
template <>
struct Pub<3> {
  union {
    double q64[4];
    struct {
      float4 q32;  // q.x, q.y, q.z, 0
      float4 d32;  // delta.x, delta.y, delta.z, 0
    } p;
  };
};

template <int D>
__device__ __forceinline__ void load_pub32(const Pub<D>* p, float* q, float* dd) {
  if constexpr (D == 2) {
    float4 a = p->p32;
    q[0] = a.x; q[1] = a.y; dd[0] = a.z; dd[1] = a.w;
  } else {
    float4 a = p->p.q32, b = p->p.d32;
    q[0] = a.x; q[1] = a.y; q[2] = a.z; dd[0] = b.x; dd[1] = b.y; dd[2] = b.z;
  }
}

template <int D>
__device__ __forceinline__ void store_pub32(Pub<D>* p, const float* q, const float* dd) {
  if constexpr (D == 2) {
    p->p32 = make_float4(q[0], q[1], dd[0], dd[1]);
  } else {
    p->p.q32 = make_float4(q[0], q[1], q[2], 0.0f);
    p->p.d32 = make_float4(dd[0], dd[1], dd[2], 0.0f);
  }
}

template <int D>
__device__ __forceinline__ void load_pub64(const Pub<D>* p, double* q) {
  if constexpr (D == 2) {
    double2 a = *reinterpret_cast<const double2*>(p->q64);
    q[0] = a.x; q[1] = a.y;
  } else {
    double2 a = *reinterpret_cast<const double2*>(p->q64);
    q[0] = a.x; q[1] = a.y; q[2] = p->q64[2];
  }
}

constexpr int kModeEval64 = 0, kModeDev = 1;

// Cell-image offsets of the FP32 pair loop, one copy per lane
// ([code * 3 + axis][32]): every lane reads its own bank, so the per-pair
// table lookup has no bank conflicts whatever codes the lanes need.
constexpr int kOffLane = 27 * 3 * 32;

// Control block written once per iteration by thread 0 of every CTA (all CTAs
// compute it from bitwise identical totals) and read by the CTA's threads.
struct Ctl {
  double dt, ratio, keep;     // FIRE step after an FP64 evaluation
  float dtf, ratiof, keepf;   // the same in FP32 for the FP32 update
  int move, mode, stop, reset, want_e, was64, status;
};


// Compensated ("float-float") sum on the FP32 pipe: TwoSum of Knuth (TAOCP
// vol. 2, 4.2.2) followed by renormalisation (Dekker 1971).  The pair
// (hi, lo) carries about 44 significant bits, so the cross-thread sums of
// |F|^2 and |v|^2 (the FIRE mixing norms) keep near-FP64 accuracy without FP64
// instructions, whose issue cost on GB300 (one warp instruction per ~32 cycles
// per SM sub-partition) would dominate an iteration if every sum used them.
// The FIRE power P = F.v, whose sign decides every step, is summed in FP64.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s = a.hi + b.hi;
  float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  float hi = s + e;
  return FF{hi, e - (hi - s)};
}
__device__ __forceinline__ FF ff_shfl_xor(FF a, int o) {
  return FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ float nmaxf(float a, float b) { return (a != a || a > b) ? a : b; }
// an FP64 value in two consecutive FP32 slots of a reduction record
__device__ __forceinline__ void put_d(float* q, double d) {
  q[0] = __int_as_float(__double2loint(d));
  q[1] = __int_as_float(__double2hiint(d));
}
__device__ __forceinline__ double get_d(const float* q) {
  return __hiloint2double(__float_as_int(q[1]), __float_as_int(q[0]));
}

// Polls of a grid-barrier wait before it gives up (each an L2 round trip plus
// a short back-off: a few seconds); a wait that runs out sets the launch's
// error word and the replica stops.
constexpr long long kGbSpinLimit = 1ll << 22;

// Grid-barrier arrival (release: the writes before it become visible to any
// thread that acquires the counter) and poll (acquire).
__device__ __forceinline__ void gb_arrive(unsigned long long* p) {
  asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ unsigned long long gb_poll(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// While the largest FP64 force exceeds this, mixed mode keeps evaluating in
// FP64 (random starts and collisions), where FP32 would overflow.
constexpr double kBigForce = 1e3;
// FP32 moves also need |v|^2 (summed over the replica) below this, so that
// velocities, powers and their float-float sums stay inside the FP32 range
constexpr double kBigV2 = 1e30;

// MEM: 0 = list in global memory, neighbour positions gathered from the owner
// CTA's shared memory (DSMEM); 1 = list staged in shared memory, DSMEM
// gathers; 2 = list staged and, every iteration, the positions of all CTAs
// that own neighbours copied into the local shared memory, so the force loop
// reads local shared memory only.
// TPA: threads per atom in the force phase.  With TPA > 1 (one atom per
// thread group of TPA adjacent lanes, APT = 1, per-atom state in global
// memory) each lane of the group visits every TPA-th list entry and the group
// sums its partial forces by shuffles in a fixed order; the other phases keep
// one thread per atom.  It halves the serial pair chain of each thread and
// doubles the warps that hide its latency.
// GB: the C CTAs of a replica are consecutive blocks of a cooperative launch
// (no thread-block cluster) and synchronise through a barrier in global
// memory (MinArgs::gb_bar), with their reduction partials in global memory;
// only the global-record staging modes (0, 3).  A cooperative launch keeps
// every CTA resident, so the replicas' CTAs are not bound to the per-GPC
// placement of clusters.
template <int D, bool MIXED, int APT, int MEM, int TPA, bool GB>
__global__ void __launch_bounds__((minimize_is_lean(D, APT) || TPA > 1) ? 1024 : 512, 1)
    k_minimize(MinArgs A) {
  static_assert(!GB || MEM == 0 || MEM == 3, "grid barriers need global neighbour records");
  cg::cluster_group cl = cg::this_cluster();
  const int C = GB ? A.gb_C : (int)cl.num_blocks();
  const int rank = GB ? (int)(blockIdx.x % (unsigned)C) : (int)cl.block_rank();
  const int ri = A.work[blockIdx.x / C];
  const RepGeom& g = A.geom[ri];
  RepState* st = A.state + ri;
  const int n = g.n, npc = g.npc;
  const int lo = rank * npc;
  const int cnt = max(0, min(npc, n - lo));
  const int64_t base = g.off + lo;  // global index of local slot 0
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = (nthr + 31) >> 5;
  const int64_t N = A.ntot;
  const int lstride = A.npc_launch;
  constexpr bool LSM = MEM >= 1;                // list rows staged in shared memory
  constexpr bool GREC = MEM == 0 || MEM == 3;   // neighbour records from global memory
  Pub<D>* pubg = reinterpret_cast<Pub<D>*>(A.pubg);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  Pub<D>* pub = reinterpret_cast<Pub<D>*>(smem_raw);  // MEM 2: whole replica, else own atoms
  // Mode 0 keeps the records of the CTA's own atoms in the global record
  // array only: the shared memory they would take is left to L1, which holds
  // the gathered neighbour records while the lists stream past.
  constexpr bool OWN_G = MEM == 0;
  Pub<D>* mine = MEM == 2 ? pub + lo : (OWN_G ? pubg + base : pub);
  const int pub_len = MEM == 2 ? A.nrep_launch : (OWN_G ? 0 : lstride);
  double* sred = reinterpret_cast<double*>(smem_raw + sizeof(Pub<D>) * pub_len);  // [kNumRed]
  // this CTA's reduction partials: shared memory (read by the other CTAs of
  // the cluster through DSMEM), or a global slot per (replica, rank) with GB
  double* red = GB ? A.gb_part + ((int64_t)ri * kMaxCluster + rank) * kNumRed : sred;
  double* wred = sred + kNumRed;                                                  // [32][kNumRed]
  double* off64 = wred + 32 * kNumRed;                                            // [27][3]
  float* off32 = reinterpret_cast<float*>(off64 + 27 * 3);                        // [27][3]
  float* off32l = off32 + 27 * 3 + 3;                                             // [27*3][32]
  PairCoef* coef = reinterpret_cast<PairCoef*>(off32l + kOffLane);                // [nt*nt]
  uint32_t* lst = reinterpret_cast<uint32_t*>(coef + A.nt * A.nt);                // [cap][lstride]
  __shared__ Pub<D>* rpub[kMaxCluster];
  __shared__ double* rred[kMaxCluster];
  __shared__ Ctl ctl;
  __shared__ double shv[4];
  __shared__ unsigned need;  // MEM 2: bit r set if rank r owns neighbours of this CTA
  __shared__ int gb_abort;   // GB: a barrier of this CTA ran out of spins
  if (tid == 0) {
    need = 0u;
    gb_abort = 0;
  }
  __syncthreads();
  // Barrier over the replica's CTAs: the cluster barrier, or with GB an
  // arrival counter in global memory (64 bits per replica, zeroed by the host
  // before every launch): the k-th barrier of a launch ends when the counter
  // reaches k C.  Thread 0 arrives with a release reduction (after the CTA
  // barrier, so it publishes the writes of every thread of the CTA) and polls
  // with acquire loads, at most kGbSpinLimit times.
  unsigned long long* gctr = GB ? reinterpret_cast<unsigned long long*>(A.gb_bar) + ri : nullptr;
  unsigned long long gb_target = 0;  // thread 0: arrivals that end the next barrier
  auto csync = [&]() {
    if constexpr (GB) {
      __syncthreads();
      if (tid == 0) {
        gb_target += (unsigned long long)C;
        gb_arrive(gctr);
        long long spins = 0;
        while (gb_poll(gctr) < gb_target) {
          if (++spins > kGbSpinLimit) {
            gb_abort = 1;
            atomicExch(A.gb_err, 1);
            break;
          }
          if (spins > 32) __nanosleep(32);
        }
      }
      __syncthreads();
    } else {
      cl.sync();
    }
  };

  // ---- set-up: geometry (tilt from the kernel-written state), tables ----
  double H[9], Hb[9];
  const bool HIST = A.hist != nullptr;  // uniform: a launch has a table or not
#pragma unroll
  for (int k = 0; k < 9; k++) H[k] = HIST ? st->Hc[k] : g.H[k];
  if (!HIST) H[1] = st->tilt;
#pragma unroll
  for (int k = 0; k < 9; k++) Hb[k] = HIST ? st->Hb[k] : 0.0;
  const int ncode = D == 2 ? 9 : 27;
  auto make_tables = [&]() {
    if (tid < ncode) {
      double o[3];
      cell_offset<D>(H, g.nc, tid, o);
      for (int k = 0; k < D; k++) {
        off64[tid * 3 + k] = o[k];
        off32[tid * 3 + k] = (float)o[k];
      }
    }
    for (int i = tid; i < ncode * 32; i += nthr) {
      double o[3];
      cell_offset<D>(H, g.nc, i >> 5, o);
      for (int k = 0; k < D; k++) off32l[((i >> 5) * 3 + k) * 32 + (i & 31)] = (float)o[k];
    }
  };
  make_tables();
  for (int k = tid; k < A.nt * A.nt; k += nthr) coef[k] = A.coef[k];
  if (tid < C) {
    if constexpr (GB) {
      rpub[tid] = nullptr;
      rred[tid] = A.gb_part + ((int64_t)ri * kMaxCluster + tid) * kNumRed;
    } else {
      rpub[tid] = cl.map_shared_rank(pub, tid);
      rred[tid] = cl.map_shared_rank(red, tid);
    }
  }
  const FireDev fp = A.fire;
  // ---- the replica's job: nsteps fine steps (affine dgamma + minimisation) ----
  int64_t step = st->step;
  const int64_t nsteps = st->nsteps;
  const bool first_noaffine = st->first_noaffine != 0;
  const bool want_snap = st->want_snap != 0;
  const double dgam = st->dgamma;
  int phase = st->phase;  // 0: the next step has not started, 1: FIRE in progress
  double tilt_b = st->tilt_b;  // changes when the kernel rebuilds the list
  // FIRE scalars (meaningful in thread 0 only)
  double dt = st->dt, alpha = st->alpha;
  float dtf = (float)dt, alphaf = (float)alpha;  // mixed mode keeps these in FP32
  int npos = st->npos;
  int64_t iters = st->iters, evals = st->evals64, evals32 = st->evals32;
  int64_t launch_iters = 0;
  int64_t acc_it = st->acc_iters, acc64 = st->acc64, acc32 = st->acc32;
  int kreb = st->kreb;
  double vol = D == 2 ? H[0] * H[3] : H[0] * H[4] * H[8];
  bool want_e = MIXED;  // mixed: every FP64 evaluation also gives E and tau
  float wmaxf = 0.0f;   // max |x_ref - x_b| at the last FP64 evaluation (mixed)
  // mixed: true while A.v holds the current velocity in FP64 (moves after FP64
  // evaluations), false while the FP32 registers v32 do (moves after FP32 ones)
  bool v64 = true;
  double gamma_term = 0.0;
  float gamma_termf = 0.0f;
  const float skinf = (float)A.skin;
  const float tolf = (float)fp.tol, ratio_f = (float)fp.ref_ratio, dmax_f = (float)fp.ref_dmax;
  const float f_incf = (float)fp.f_inc, f_decf = (float)fp.f_dec, f_alphaf = (float)fp.f_alpha;
  const float dt_maxf = (float)fp.dt_max, dt_minf = (float)fp.dt_min, alpha0f = (float)fp.alpha0;
  int status = kStatusRunning;
  double E = 0.0, W = 0.0, fmx = 0.0;

  // Per-atom state.  With few atoms per thread it lives in registers; with
  // more ("lean" launches: 4 or 8 atoms per thread, 2 or more in 3D)
  // registers would spill, so it lives in global memory (L2) and only the
  // atom being processed is in registers: FP32 reference position, displacement, velocity, reference
  // force and the force used by the update, and the FP64 force.
  constexpr bool LEAN = minimize_is_lean(D, APT) || TPA > 1;
  static_assert(TPA == 1 || APT == 1, "split force phase runs one atom per thread group");
  // pair-loop unrolling: lean launches keep more list and record loads in
  // flight per thread (they stream the lists from HBM)
  constexpr int kPairUnroll = LEAN ? 8 : 4;
  constexpr int AR = LEAN ? 1 : APT;
  int ty[APT];
  float q32[AR][3], d32[AR][3], v32[AR][3], fr32[AR][3], Fu[AR][3];
  double F[AR][3];
  float* const l32 = A.lean32;   // [5][3][ntot]: q, delta, v, f_ref, f_used
  double* const l64 = A.lean64;  // [3][ntot]: FP64 force
  auto Q = [&](int k, int c) -> float& {
    if constexpr (LEAN) return l32[(0 * 3 + c) * N + base + tid + k * nthr];
    else return q32[k][c];
  };
  auto Dl = [&](int k, int c) -> float& {
    if constexpr (LEAN) return l32[(1 * 3 + c) * N + base + tid + k * nthr];
    else return d32[k][c];
  };
  auto V = [&](int k, int c) -> float& {
    if constexpr (LEAN) return l32[(2 * 3 + c) * N + base + tid + k * nthr];
    else return v32[k][c];
  };
  auto FR = [&](int k, int c) -> float& {
    if constexpr (LEAN) return l32[(3 * 3 + c) * N + base + tid + k * nthr];
    else return fr32[k][c];
  };
  auto FU = [&](int k, int c) -> float& {
    if constexpr (LEAN) return l32[(4 * 3 + c) * N + base + tid + k * nthr];
    else return Fu[k][c];
  };
  auto FD = [&](int k, int c) -> double& {
    if constexpr (LEAN) return l64[c * N + base + tid + k * nthr];
    else return F[k][c];
  };
  auto pub32 = [&](int k) {  // publish the FP32 view of the record of atom slot k
    const int li = tid + k * nthr;
    float qq[3], dq[3];
#pragma unroll
    for (int c = 0; c < D; c++) {
      qq[c] = Q(k, c);
      dq[c] = Dl(k, c);
    }
    store_pub32<D>(&mine[li], qq, dq);
    if (GREC && !OWN_G) store_pub32<D>(&pubg[base + li], qq, dq);
  };
#pragma unroll
  for (int k = 0; k < APT; k++) {
    int li = tid + k * nthr;
    ty[k] = 0;
    if (!LEAN || li < cnt) {
#pragma unroll
      for (int c = 0; c < 3; c++) Q(k, c) = Dl(k, c) = V(k, c) = FR(k, c) = FU(k, c) = 0.0f;
    }
    if (li < cnt) {
      int64_t gi = base + li;
      ty[k] = A.type[gi];
      if (MIXED && phase == 1)
        for (int c = 0; c < D; c++) V(k, c) = (float)A.v[c * N + gi];
      if (LSM) {
        const int nn = A.nnb[gi];
        const uint32_t* row = A.nb + g.nb_off + lo + li;
        unsigned m = 0u;
        for (int j = 0; j < nn; j++) {
          uint32_t ent = __ldg(row + (int64_t)j * n);
          lst[j * lstride + li] = ent;
          m |= 1u << nb_owner(ent);
        }
        if (MEM == 2 && m) atomicOr(&need, m);
      }
    }
  }
  auto publish64 = [&](int k) {
    int li = tid + k * nthr;
    int64_t gi = base + li;
    double o[3];
    cell_origin<D>(H, g.nc, A.cell[gi], o);
    double* q = mine[li].q64;
    for (int c = 0; c < D; c++) q[c] = A.x[c * N + gi] - o[c];
    if (GREC && !OWN_G)
      for (int c = 0; c < D; c++) pubg[gi].q64[c] = q[c];
  };
  // record of a neighbour (owner CTA, slot) for the force phase
  auto nbrec = [&](uint32_t ent) -> const Pub<D>* {
    const int ow = nb_owner(ent), sl = nb_slot(ent);
    if (MEM == 2) return pub + ow * npc + sl;
    if (GREC) return pubg + (g.off + (int64_t)ow * npc + sl);
    return ow == rank ? mine + sl : rpub[ow] + sl;
  };
  // MEM 2: copy the records of the other CTAs that own neighbours (16-byte words)
  auto stage = [&]() {
    constexpr int Wd = sizeof(Pub<D>) / 16;
    for (int r = 0; r < C; r++) {
      if (r == rank || !((need >> r) & 1u)) continue;
      const int cr = max(0, min(npc, n - r * npc));
      const uint4* src = reinterpret_cast<const uint4*>(rpub[r] + r * npc);
      uint4* dst = reinterpret_cast<uint4*>(pub + r * npc);
      for (int w = tid; w < cr * Wd; w += nthr) dst[w] = src[w];
    }
  };
  // cluster-wide FP64 reduction of nv (<= 4) values; identical result in every CTA
  auto cluster_reduce = [&](double* v, int nv, bool is_max) {
    for (int m = 0; m < nv; m++)
      for (int o = 16; o > 0; o >>= 1) {
        double t = __shfl_xor_sync(0xffffffffu, v[m], o);
        v[m] = is_max ? fmax(v[m], t) : v[m] + t;
      }
    if (lane == 0)
      for (int m = 0; m < nv; m++) wred[warp * kNumRed + m] = v[m];
    __syncthreads();
    if (warp == 0) {
      for (int m = 0; m < nv; m++) {
        double t = lane < nwarp ? wred[lane * kNumRed + m] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
          double u = __shfl_xor_sync(0xffffffffu, t, o);
          t = is_max ? fmax(t, u) : t + u;
        }
        if (lane == 0) red[m] = t;
      }
    }
    csync();
    if (warp == 0) {
      for (int m = 0; m < nv; m++) {
        double t = lane < C ? rred[lane][m] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
          double u = __shfl_xor_sync(0xffffffffu, t, o);
          t = is_max ? fmax(t, u) : t + u;
        }
        if (lane == 0) shv[m] = t;
      }
    }
    csync();  // every CTA has read the partials before they are reused
    for (int m = 0; m < nv; m++) v[m] = shv[m];
  };

  // ---- in-kernel Verlet rebuild (the atoms keep their CTA and slot) ----
  // Called by every thread of every CTA of the cluster with x materialised.
  // Returns false (uniformly) when the host must take over: the cell grid no
  // longer covers rc + skin at the current tilt, or a list would overflow.
  auto rebuild_lists = [&]() -> bool {
    // cell grid still wide enough for the 3^d stencil at the current tilt?
    {
      const double t = H[1] / H[D + 1];
      double w = (H[0] / sqrt(1.0 + t * t)) / g.nc[0];
      w = fmin(w, H[D + 1] / g.nc[1]);
      if (D == 3) w = fmin(w, H[8] / g.nc[2]);
      if (!(w >= A.rlist)) return false;
    }
    const int32_t coff = g.cell_off;
    const int ncell = g.ncell;
    const int64_t aoff = g.off;
    // 1. wrap own atoms into the cell (by whole lattice vectors, the same
    //    shift applied to the step's start positions), new cell keys
    for (int c = rank * nthr + tid; c <= ncell; c += C * nthr) A.count[coff + c] = 0;
#pragma unroll
    for (int k = 0; k < APT; k++) {
      int li = tid + k * nthr;
      if (li >= cnt) continue;
      int64_t gi = base + li;
      double xv[3], sv[3];
      for (int c = 0; c < D; c++) xv[c] = A.x[c * N + gi];
      for (int c = D - 1; c >= 0; c--) {
        double tt = xv[c];
        for (int kk = c + 1; kk < D; kk++) tt -= H[c * D + kk] * sv[kk];
        sv[c] = tt / H[c * D + c];
      }
      int key = 0, mul = 1;
      for (int c = 0; c < D; c++) {
        double nf = floor(sv[c]);
        if (nf != 0.0)
          for (int a = 0; a <= c; a++) {
            A.x[a * N + gi] -= nf * H[a * D + c];
            A.xs[a * N + gi] -= nf * H[a * D + c];
          }
        int ic = (int)floor((sv[c] - nf) * g.nc[c]);
        ic = ic < 0 ? 0 : (ic >= g.nc[c] ? g.nc[c] - 1 : ic);
        key += ic * mul;
        mul *= g.nc[c];
      }
      A.cell[gi] = key;
      // FP32 position relative to the new cell origin, computed once per atom
      // and read by every candidate test below (the global record array is
      // free during the rebuild; the records are published again after it)
      double o[3];
      cell_origin<D>(H, g.nc, key, o);
      float qf[3] = {0.f, 0.f, 0.f}, zf[3] = {0.f, 0.f, 0.f};
      for (int c = 0; c < D; c++) qf[c] = (float)(A.x[c * N + gi] - o[c]);
      store_pub32<D>(&pubg[gi], qf, zf);
    }
    csync();
    // 2. histogram
#pragma unroll
    for (int k = 0; k < APT; k++) {
      int li = tid + k * nthr;
      if (li < cnt) atomicAdd(&A.count[coff + A.cell[base + li]], 1);
    }
    csync();
    // 3. exclusive scan (rank 0), counts become scatter cursors
    if (rank == 0) {
      int* swsum = reinterpret_cast<int*>(wred);  // [32] warp sums, [32] carry
      int& scarry = swsum[32];
      if (tid == 0) scarry = 0;
      __syncthreads();
      for (int b0 = 0; b0 < ncell; b0 += nthr) {
        const int c = b0 + tid;
        const int v = c < ncell ? A.count[coff + c] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
          int tt = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += tt;
        }
        if (lane == 31) swsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
          int ws = lane < nwarp ? swsum[lane] : 0;
          for (int o = 1; o < 32; o <<= 1) {
            int tt = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += tt;
          }
          if (lane < nwarp) swsum[lane] = ws;
        }
        __syncthreads();
        if (c < ncell) {
          A.cstart[coff + c] = scarry + (warp > 0 ? swsum[warp - 1] : 0) + incl - v;
          A.count[coff + c] = 0;
        }
        __syncthreads();
        if (tid == 0) scarry += swsum[nwarp - 1];
        __syncthreads();
      }
      if (tid == 0) A.cstart[coff + ncell] = scarry;
    }
    csync();
    // 4. scatter replica-local indices into the cells
#pragma unroll
    for (int k = 0; k < APT; k++) {
      int li = tid + k * nthr;
      if (li >= cnt) continue;
      const int key = A.cell[base + li];
      const int p = A.cstart[coff + key] + atomicAdd(&A.count[coff + key], 1);
      A.cellatoms[aoff + p] = lo + li;
    }
    csync();
    // 5. deterministic order inside each cell
    for (int c = rank * nthr + tid; c < ncell; c += C * nthr) {
      const int b = A.cstart[coff + c], e = A.cstart[coff + c + 1];
      for (int i = b + 1; i < e; i++) {
        const int v = A.cellatoms[aoff + i];
        int j = i - 1;
        while (j >= b && A.cellatoms[aoff + j] > v) {
          A.cellatoms[aoff + j + 1] = A.cellatoms[aoff + j];
          j--;
        }
        A.cellatoms[aoff + j + 1] = v;
      }
    }
    csync();
    // 6. Verlet rows of the own atoms (same test as the host-side build),
    //    written to the global list and, when staged, to shared memory
    if (MEM == 2 && tid == 0) need = 0u;
    __syncthreads();
    double over = 0.0;
    const int ncode = D == 2 ? 9 : 27;
#pragma unroll
    for (int k = 0; k < APT; k++) {
      int li = tid + k * nthr;
      if (li >= cnt) continue;
      const int64_t gi = base + li;
      const int il = lo + li;
      const int ci = A.cell[gi];
      int cc[3] = {ci % g.nc[0], (ci / g.nc[0]) % g.nc[1], D == 3 ? ci / (g.nc[0] * g.nc[1]) : 0};
      float qi[3], zi[3];
      load_pub32<D>(&pubg[gi], qi, zi);
      const int ti = ty[k];
      int m = 0;
      unsigned own = 0u;
      for (int code = 0; code < ncode; code++) {
        const int dx = code % 3 - 1, dy = (code / 3) % 3 - 1, dz = code / 9 - 1;
        const int nx = (cc[0] + dx + g.nc[0]) % g.nc[0];
        const int ny = (cc[1] + dy + g.nc[1]) % g.nc[1];
        const int nz = D == 3 ? (cc[2] + dz + g.nc[2]) % g.nc[2] : 0;
        const int cj = nx + g.nc[0] * (ny + g.nc[1] * nz);
        const float* of = off32 + 3 * code;
        const int b = A.cstart[g.cell_off + cj], e = A.cstart[g.cell_off + cj + 1];
        for (int p = b; p < e; p++) {
          const int jl = A.cellatoms[g.off + p];
          if (jl == il) continue;
          const int64_t gj = g.off + jl;
          float qj[3], zj[3];
          load_pub32<D>(&pubg[gj], qj, zj);
          float s2 = 0.0f;
          for (int c = 0; c < D; c++) {
            float d = (qj[c] - qi[c]) + of[c];
            s2 = fmaf(d, d, s2);
          }
          const int tj = A.type[gj];
          if (s2 < A.rl2f[ti * A.nt + tj]) {
            if (m < A.cap) {
              const uint32_t ent = encode_nb(jl % npc, jl / npc, code, tj);
              A.nb[g.nb_off + (int64_t)m * n + il] = ent;
              if (LSM && m < A.cap) lst[m * lstride + li] = ent;
              own |= 1u << (jl / npc);
            }
            m++;
          }
        }
      }
      A.nnb[gi] = m < A.cap ? m : A.cap;
      if (m > A.cap) over = 1.0;
      if (MEM == 2 && own) atomicOr(&need, own);
      for (int c = 0; c < D; c++) A.xb[c * N + gi] = A.x[c * N + gi];
    }
    double ov[1] = {over};
    cluster_reduce(ov, 1, true);  // also orders the list writes before their use
    return ov[0] == 0.0 && !(GB && gb_abort);
  };


  for (;;) {
    if (step >= nsteps) {
      status = AQS_OK;
      break;
    }
    if (phase == 0) {
      // ---- start of a fine step: affine map (Eq. 16) unless it is the
      // level-II chain's first minimisation, then a fresh FIRE ----
      const bool affine = !(step == 0 && first_noaffine);
#pragma unroll
      for (int k = 0; k < APT; k++) {
        int li = tid + k * nthr;
        if (li >= cnt) continue;
        int64_t gi = base + li;
        if (affine && HIST) {
          // deformation history: x <- M x (upper triangular), the list-build
          // positions alike
          const double* M = A.hist + ((int64_t)ri * A.hist_stride + step) * kHistFields;
          for (int a = 0; a < D; a++) {
            double xa = M[a * 3 + a] * A.x[a * N + gi], ba = M[a * 3 + a] * A.xb[a * N + gi];
            for (int c = a + 1; c < D; c++) {
              xa = fma(M[a * 3 + c], A.x[c * N + gi], xa);
              ba = fma(M[a * 3 + c], A.xb[c * N + gi], ba);
            }
            A.x[a * N + gi] = xa;
            A.xb[a * N + gi] = ba;
          }
        } else if (affine) {
          A.x[gi] = fma(dgam, A.x[N + gi], A.x[gi]);
          A.xb[gi] = fma(dgam, A.xb[N + gi], A.xb[gi]);
          if (A.warm_u) {
            // learned start: F r_k + dgamma u (caller-order prediction)
            const float* u = A.warm_u + (g.off + A.perm[gi]) * D;
            for (int c = 0; c < D; c++) A.x[c * N + gi] = fma(dgam, (double)u[c], A.x[c * N + gi]);
          }
        }
        for (int c = 0; c < D; c++) {
          A.v[c * N + gi] = 0.0;
          A.xs[c * N + gi] = A.x[c * N + gi];
          V(k, c) = 0.0f;
          Dl(k, c) = 0.0f;
        }
      }
      if (affine && HIST) {
        const double* Hn = A.hist + ((int64_t)ri * A.hist_stride + step) * kHistFields + 9;
        for (int a = 0; a < D; a++)
          for (int c = 0; c < D; c++) H[a * D + c] = Hn[a * 3 + c];
        vol = D == 2 ? H[0] * H[3] : H[0] * H[4] * H[8];
      } else if (affine) {
        H[1] = fma(dgam, H[D + 1], H[1]);
      }
      dt = fp.dt0;
      alpha = fp.alpha0;
      dtf = (float)dt;
      alphaf = (float)alpha;
      npos = 0;
      iters = evals = evals32 = 0;
      want_e = MIXED;
      v64 = true;
      phase = 1;
      make_tables();
    }
    gamma_term = HIST ? affine_change<D>(H, Hb) * A.rlist : fabs(H[1] - tilt_b) / H[D + 1] * A.rlist;
    gamma_termf = (float)gamma_term;
#pragma unroll
    for (int k = 0; k < APT; k++)
      if (tid + k * nthr < cnt) publish64(k);
    int mode = kModeEval64;
    csync();

    for (;;) {
      if (MEM == 2) {
        stage();
        __syncthreads();
      }
    // ================= force phase =================
    double r[kNumRed];
#pragma unroll
    for (int m = 0; m < kNumRed; m++) r[m] = 0.0;
    float rf[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // DEV: fmax^2, -, |F|^2, |v|^2, max|delta|^2
    double rp = 0.0;  // DEV: the FIRE power P = F.v, summed in FP64
    // 3D lean launches walk their atoms one at a time (the per-atom state is in
    // global memory, ~100 list entries give each atom's loop its own
    // parallelism, and unrolling over atoms only lengthens live ranges at 64
    // registers: 4 % faster); 2D lists are short, there the unrolled atoms
    // are the parallelism
#pragma unroll ((LEAN && D == 3) ? 1 : APT)
    for (int k = 0; k < APT; k++) {
      if constexpr (!LEAN) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
          F[k][c] = 0.0;
          Fu[k][c] = 0.0f;
        }
      }
      // force-phase atom of this thread: li (TPA > 1: shared by TPA lanes, this
      // lane's list entries are those with j = h mod TPA)
      const int li = TPA > 1 ? tid / TPA : tid + k * nthr;
      const int h = TPA > 1 ? (tid & (TPA - 1)) : 0;
      if (li >= cnt) continue;
      int64_t gi = base + li;
      const uint32_t* row = A.nb + g.nb_off + lo + li;
      const int nn = A.nnb[gi];
      const int ti = (TPA > 1 || (LEAN && D == 3)) ? A.type[gi] : ty[k];
      // per-atom state of this atom (written by the group's first lane)
      auto FDa = [&](int c) -> double& {
        if constexpr (TPA > 1) return l64[c * N + gi];
        else return FD(k, c);
      };
      auto FRa = [&](int c) -> float& {
        if constexpr (TPA > 1) return l32[(3 * 3 + c) * N + gi];
        else return FR(k, c);
      };
      auto FUa = [&](int c) -> float& {
        if constexpr (TPA > 1) return l32[(4 * 3 + c) * N + gi];
        else return FU(k, c);
      };
      auto Qa = [&](int c) -> float& {
        if constexpr (TPA > 1) return l32[(0 * 3 + c) * N + gi];
        else return Q(k, c);
      };
      auto Va = [&](int c) -> float& {
        if constexpr (TPA > 1) return l32[(2 * 3 + c) * N + gi];
        else return V(k, c);
      };
      // lanes of this atom's group (a subset of the warp: the groups of a
      // warp need not all have an atom)
      const unsigned gmask = TPA > 1 ? (((1u << TPA) - 1u) << (lane & ~(TPA - 1))) : 0xffffffffu;
      if (mode == kModeEval64) {
        double qi[3], e = 0.0, w = 0.0, Fk[3] = {0.0, 0.0, 0.0};
        load_pub64<D>(&mine[li], qi);
#pragma unroll 4
        for (int j = h; j < nn; j += TPA) {
          uint32_t ent = LSM ? lst[j * lstride + li] : __ldcs(row + (int64_t)j * n);
          double qj[3], d[3];
          load_pub64<D>(nbrec(ent), qj);
          const double* of = off64 + 3 * nb_code(ent);
#pragma unroll
          for (int c = 0; c < D; c++) d[c] = (qj[c] - qi[c]) + of[c];
          pair64<D>(coef[ti * A.nt + nb_type(ent)], d, Fk, want_e, e, w);
        }
        if constexpr (TPA > 1) {
#pragma unroll
          for (int o = 1; o < TPA; o <<= 1)
#pragma unroll
            for (int c = 0; c < D; c++) Fk[c] += __shfl_xor_sync(gmask, Fk[c], o);
        }
        r[6] += e;
        r[7] += w;
        if (h == 0) {
#pragma unroll
          for (int c = 0; c < D; c++) FDa(c) = Fk[c];
          double f2 = 0.0, pv = 0.0, v2 = 0.0, u2 = 0.0;
#pragma unroll
          for (int c = 0; c < D; c++) {
            double vc = (MIXED && !v64) ? (double)Va(c) : A.v[c * N + gi];
            f2 = fma(Fk[c], Fk[c], f2);
            pv = fma(Fk[c], vc, pv);
            v2 = fma(vc, vc, v2);
            double u = A.x[c * N + gi] - A.xb[c * N + gi];
            u2 = fma(u, u, u2);
          }
          if (MIXED) {
#pragma unroll
            for (int c = 0; c < D; c++) {
              FRa(c) = (float)Fk[c];
              FUa(c) = (float)Fk[c];
              Qa(c) = (float)qi[c];
            }
          }
          r[0] = nmax(r[0], f2);
          r[1] += pv;
          r[2] += f2;
          r[3] += v2;
          r[5] = nmax(r[5], u2);
        }
      } else {
        float qi[3], di[3], f[3] = {0.f, 0.f, 0.f};
        load_pub32<D>(&mine[li], qi, di);
        auto pair_loop = [&](auto coef_of) {
#pragma unroll kPairUnroll
          for (int j = h; j < nn; j += TPA) {
            uint32_t ent = LSM ? lst[j * lstride + li] : __ldcs(row + (int64_t)j * n);
            float qj[3], dj[3], d0[3], e[3];
            load_pub32<D>(nbrec(ent), qj, dj);
            const float* of = off32l + 3 * 32 * nb_code(ent) + lane;
#pragma unroll
            for (int c = 0; c < D; c++) {
              d0[c] = (qj[c] - qi[c]) + of[c * 32];
              e[c] = dj[c] - di[c];
            }
            pair_dev<D>(coef_of(nb_type(ent)), d0, e, f);
          }
        };
        if (A.nt <= 2) {
          // the two species rows of this atom in registers
          const Coef32 c0 = coef32(coef[ti * A.nt]);
          const Coef32 c1 = A.nt > 1 ? coef32(coef[ti * A.nt + 1]) : c0;
          pair_loop([&](int tj) { return tj ? c1 : c0; });
        } else {
          pair_loop([&](int tj) { return coef32(coef[ti * A.nt + tj]); });
        }
        if constexpr (TPA > 1) {
#pragma unroll
          for (int o = 1; o < TPA; o <<= 1)
#pragma unroll
            for (int c = 0; c < D; c++) f[c] += __shfl_xor_sync(gmask, f[c], o);
        }
        if (h == 0) {
          float f2 = 0.f, v2 = 0.f, dd = 0.f;
          double pv = 0.0;  // FP32 products are exact in FP64
#pragma unroll
          for (int c = 0; c < D; c++) {
            const float fu = FRa(c) + f[c];
            const float vk = Va(c);
            FUa(c) = fu;
            f2 = fmaf(fu, fu, f2);
            pv = fma((double)fu, (double)vk, pv);
            v2 = fmaf(vk, vk, v2);
            dd = fmaf(di[c], di[c], dd);  // the published displacement
          }
          rf[0] = nmaxf(rf[0], f2);
          rp += pv;
          rf[2] += f2;
          rf[3] += v2;
          rf[4] = nmaxf(rf[4], dd);
        }
      }
    }

    // ================= reduction (fixed order; FP64, or float-float norms and FP64 power) =================
    const bool fast = MIXED && mode == kModeDev;  // uniform in the cluster
    double T[kNumRed];  // FP64 totals (valid in warp 0)
    float Tf[5];        // DEV totals (valid in warp 0)
    double Pd = 0.0;    // DEV: the FIRE power, FP64 (valid in warp 0)
    if (!fast) {
#pragma unroll
      for (int m = 0; m < kNumRed; m++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          double t = __shfl_xor_sync(0xffffffffu, r[m], o);
          r[m] = is_max_slot(m) ? nmax(r[m], t) : r[m] + t;
        }
      }
      if (lane == 0)
        for (int m = 0; m < kNumRed; m++) wred[warp * kNumRed + m] = r[m];
      __syncthreads();
      if (warp == 0) {
#pragma unroll
        for (int m = 0; m < kNumRed; m++) {
          double t = lane < nwarp ? wred[lane * kNumRed + m] : 0.0;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            double u = __shfl_xor_sync(0xffffffffu, t, o);
            t = is_max_slot(m) ? nmax(t, u) : t + u;
          }
          if (lane == 0) red[m] = t;
        }
      }
      csync();  // (A) partials of every CTA visible; all force phases done
      if (warp == 0) {
#pragma unroll
        for (int m = 0; m < kNumRed; m++) {
          double t = lane < C ? rred[lane][m] : 0.0;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            double u = __shfl_xor_sync(0xffffffffu, t, o);
            t = is_max_slot(m) ? nmax(t, u) : t + u;
          }
          T[m] = t;
        }
      }
    } else {
      float m0 = rf[0], m4 = rf[4];
      double sp = rp;
      FF sf{rf[2], 0.f}, sv{rf[3], 0.f};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        m0 = nmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
        m4 = nmaxf(m4, __shfl_xor_sync(0xffffffffu, m4, o));
        sp += __shfl_xor_sync(0xffffffffu, sp, o);
        sf = ff_add(sf, ff_shfl_xor(sf, o));
        sv = ff_add(sv, ff_shfl_xor(sv, o));
      }
      float* w32 = reinterpret_cast<float*>(wred);
      if (lane == 0) {
        float* q = w32 + warp * 8;
        q[0] = m0; q[1] = m4; put_d(q + 2, sp);
        q[4] = sf.hi; q[5] = sf.lo; q[6] = sv.hi; q[7] = sv.lo;
      }
      __syncthreads();
      // butterfly over 8-float records (max, max, the FP64 power, two
      // float-float sums)
      auto reduce8 = [&](const float* q, bool valid, float* out) {
        float a0 = valid ? q[0] : 0.f, a4 = valid ? q[1] : 0.f;
        double bp = valid ? get_d(q + 2) : 0.0;
        FF bf{valid ? q[4] : 0.f, valid ? q[5] : 0.f};
        FF bv{valid ? q[6] : 0.f, valid ? q[7] : 0.f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a0 = nmaxf(a0, __shfl_xor_sync(0xffffffffu, a0, o));
          a4 = nmaxf(a4, __shfl_xor_sync(0xffffffffu, a4, o));
          bp += __shfl_xor_sync(0xffffffffu, bp, o);
          bf = ff_add(bf, ff_shfl_xor(bf, o));
          bv = ff_add(bv, ff_shfl_xor(bv, o));
        }
        out[0] = a0; out[1] = a4; put_d(out + 2, bp);
        out[4] = bf.hi; out[5] = bf.lo; out[6] = bv.hi; out[7] = bv.lo;
      };
      float* red32 = reinterpret_cast<float*>(red);
      if (warp == 0) {
        float o8[8];
        reduce8(w32 + lane * 8, lane < nwarp, o8);
        if (lane == 0)
          for (int m = 0; m < 8; m++) red32[m] = o8[m];
      }
      csync();  // (A) partials of every CTA visible; all force phases done
      if (warp == 0) {
        float o8[8];
        const float* rq = lane < C ? reinterpret_cast<const float*>(rred[lane]) : red32;
        reduce8(rq, lane < C, o8);
        Tf[0] = o8[0];
        Tf[4] = o8[1];
        Pd = get_d(o8 + 2);
        Tf[1] = (float)Pd;
        Tf[2] = o8[4] + o8[5];
        Tf[3] = o8[6] + o8[7];
      }
    }

    // ================= decisions (thread 0; identical in every CTA) =================
    if (warp == 0 && lane == 0) {
      const bool was64 = mode == kModeEval64;
      int next = -1;  // -1: FIRE move; else no-move re-evaluation in that mode
      bool stop = false;
      Ctl c;
      c.reset = 0;
      if (GB && gb_abort) {
        status = AQS_ERR_TIMEOUT;
        c.stop = 1;
        c.move = 0;
        c.dtf = c.ratiof = 0.f;
        c.keepf = 1.f;
        c.dt = c.ratio = 0.0;
        c.keep = 1.0;
      } else if (MIXED) {
        float fm, umax, P, F2, V2;
        bool finite;
        if (was64) {
          evals++;
          acc64++;
          fmx = sqrt(T[0]);
          fm = (float)fmx;
          finite = (T[0] < INFINITY) && (T[2] < INFINITY) && (T[1] == T[1]) &&
                   (!want_e || fabs(T[6]) < INFINITY);
          umax = sqrtf((float)T[5]);
          wmaxf = umax;
          P = (float)T[1];
          F2 = (float)T[2];
          V2 = (float)T[3];
        } else {
          evals32++;
          acc32++;
          fm = sqrtf(Tf[0]);
          finite = (Tf[0] < INFINITY) && (Tf[2] < INFINITY) && (Pd == Pd);
          umax = wmaxf + sqrtf(Tf[4]);
          P = Tf[1];
          F2 = Tf[2];
          V2 = Tf[3];
        }
        if (2.0f * umax + gamma_termf > skinf) {
          status = kStatusRebuild;  // forces of this pass may miss pairs: discard
          stop = true;
        } else if (!finite) {
          if (!was64) next = kModeEval64;
          else { status = AQS_ERR_NONFINITE; stop = true; }
        } else if (was64 && fmx < fp.tol) {  // the convergence test, FP64
          E = 0.5 * T[6];
          W = 0.5 * T[7] / vol;
          status = AQS_OK;
          stop = true;
        } else if (!was64 && (fm < tolf || sqrtf(Tf[4]) > fminf(ratio_f * fm, dmax_f))) {
          next = kModeEval64;  // new FP64 reference at the current positions
        } else if (iters >= fp.max_iter) {
          status = AQS_ERR_NOT_CONVERGED;
          stop = true;
        } else if (launch_iters >= A.launch_budget) {
          stop = true;  // status stays "running": the next launch resumes
        }
        c.stop = stop;
        c.move = !stop && next < 0;
        c.dtf = dtf;
        c.ratiof = 0.f;
        c.keepf = 1.f;
        c.dt = (double)dtf;
        c.ratio = 0.0;
        c.keep = 1.0;
        if (c.move) {
          if (was64 ? (T[1] >= 0.0) : (Pd >= 0.0)) {  // the FIRE power's sign, FP64
            npos++;
            if (npos > fp.n_min) {
              dtf = fminf(dtf * f_incf, dt_maxf);
              alphaf *= f_alphaf;
            }
          } else {
            npos = 0;
            dtf = fmaxf(dtf * f_decf, dt_minf);
            alphaf = alpha0f;
            c.reset = 1;
          }
          if (was64) {
            // after an FP64 evaluation the sums may exceed the FP32 range
            const double d = dtf, a = alphaf;
            const double vn2 = c.reset ? d * d * T[2] : T[3] + 2.0 * d * T[1] + d * d * T[2];
            c.dt = d;
            c.ratio = a * sqrt(vn2 / T[2]);
            c.keep = 1.0 - a;
          } else {
            const float vn2 = c.reset ? dtf * dtf * F2 : V2 + 2.0f * dtf * P + dtf * dtf * F2;
            c.dtf = dtf;
            c.ratiof = alphaf * sqrtf(vn2 / F2);
            c.keepf = 1.0f - alphaf;
          }
          iters++;
          acc_it++;
          mode = (was64 && (fmx > kBigForce || T[3] > kBigV2)) ? kModeEval64 : kModeDev;
        } else if (!stop) {
          mode = kModeEval64;
        }
      } else {
        evals++;
        acc64++;
        fmx = sqrt(T[0]);
        const bool finite = (T[0] < INFINITY) && (T[2] < INFINITY) && (T[1] == T[1]) &&
                            (!want_e || (fabs(T[6]) < INFINITY));
        const double umax = sqrt(T[5]);
        if (2.0 * umax + gamma_term > A.skin) {
          status = kStatusRebuild;
          stop = true;
        } else if (!finite) {
          status = AQS_ERR_NONFINITE;
          stop = true;
        } else if (fmx < fp.tol) {
          if (want_e) {
            E = 0.5 * T[6];
            W = 0.5 * T[7] / vol;
            status = AQS_OK;
            stop = true;
          } else {
            want_e = true;  // one more FP64 pass at the same positions for E and tau
            next = kModeEval64;
          }
        } else if (iters >= fp.max_iter) {
          status = AQS_ERR_NOT_CONVERGED;
          stop = true;
        } else if (launch_iters >= A.launch_budget) {
          stop = true;
        }
        c.stop = stop;
        c.move = !stop && next < 0;
        c.dt = dt;
        c.ratio = 0.0;
        c.keep = 1.0;
        if (c.move) {
          const double P = T[1], F2 = T[2], V2 = T[3];
          if (P >= 0.0) {
            npos++;
            if (npos > fp.n_min) {
              dt = fmin(dt * fp.f_inc, fp.dt_max);
              alpha *= fp.f_alpha;
            }
          } else {
            npos = 0;
            dt = fmax(dt * fp.f_dec, fp.dt_min);
            alpha = fp.alpha0;
            c.reset = 1;
          }
          // |v + dt F| after the Euler step, from the reductions already made
          const double vn2 = c.reset ? dt * dt * F2 : V2 + 2.0 * dt * P + dt * dt * F2;
          c.dt = dt;
          c.ratio = alpha * sqrt(vn2 / F2);
          c.keep = 1.0 - alpha;
          iters++;
          acc_it++;
        }
        mode = kModeEval64;
        c.dtf = c.ratiof = 0.f;
        c.keepf = 1.f;
      }
      c.mode = mode;
      c.want_e = want_e;
      c.was64 = was64;
      c.status = status;
      ctl = c;
    }
    __syncthreads();
    const Ctl c = ctl;
    mode = c.mode;
    want_e = c.want_e;
    status = c.status;
    if (c.move) launch_iters++;  // uniform in every thread
    if (c.stop) break;

    if (c.move) {
      // ================= FIRE update =================
      if (MIXED && c.was64) {
        // step after an FP64 evaluation: FP64 arithmetic and an FP64 velocity
        // (forces and velocities may exceed the FP32 range)
#pragma unroll
        for (int k = 0; k < APT; k++) {
          int li = tid + k * nthr;
          if (li >= cnt) continue;
          const int64_t gv = base + li;
          double sv[3], mx = 0.0;
#pragma unroll
          for (int cc = 0; cc < D; cc++) {
            double vc = c.reset ? 0.0 : (v64 ? A.v[cc * N + gv] : (double)V(k, cc));
            const double fk = FD(k, cc);
            vc = fma(c.keep, fma(c.dt, fk, vc), c.ratio * fk);
            A.v[cc * N + gv] = vc;
            V(k, cc) = (float)vc;  // used only once |v|^2 < kBigV2
            sv[cc] = c.dt * vc;
            mx = fmax(mx, fabs(sv[cc]));
          }
          double scale = 1.0;
          if (mx > 0.5 * fp.max_step) {
            double l2 = 0.0;
#pragma unroll
            for (int cc = 0; cc < D; cc++) l2 += (sv[cc] / mx) * (sv[cc] / mx);
            double len = mx * sqrt(l2);
            if (len > fp.max_step) scale = fp.max_step / len;
          }
#pragma unroll
          for (int cc = 0; cc < D; cc++) Dl(k, cc) = (float)((double)Dl(k, cc) + scale * sv[cc]);
          if (c.mode == kModeDev) {
            pub32(k);
          } else {  // the next evaluation is FP64: fold delta into x and publish it
            int64_t gi = base + li;
            for (int cc = 0; cc < D; cc++) {
              A.x[cc * N + gi] += (double)Dl(k, cc);
              Dl(k, cc) = 0.0f;
            }
            publish64(k);
          }
        }
        v64 = true;
      } else if (MIXED) {
        v64 = false;
        const float dtf = c.dtf, kf = c.keepf, rf = c.ratiof;
        const float ms = (float)fp.max_step;
#pragma unroll
        for (int k = 0; k < APT; k++) {
          int li = tid + k * nthr;
          if (li >= cnt) continue;
          float sv[3], mx = 0.0f;
#pragma unroll
          for (int cc = 0; cc < D; cc++) {
            float vc = c.reset ? 0.0f : V(k, cc);
            const float fu = FU(k, cc);
            vc = fmaf(kf, fmaf(dtf, fu, vc), rf * fu);
            V(k, cc) = vc;
            sv[cc] = dtf * vc;
            mx = fmaxf(mx, fabsf(sv[cc]));
          }
          float scale = 1.0f;
          if (mx > 0.5f * ms) {
            float l2 = 0.0f;
#pragma unroll
            for (int cc = 0; cc < D; cc++) l2 = fmaf(sv[cc] / mx, sv[cc] / mx, l2);
            float len = mx * sqrtf(l2);
            if (len > ms) scale = ms / len;
          }
#pragma unroll
          for (int cc = 0; cc < D; cc++) Dl(k, cc) = fmaf(scale, sv[cc], Dl(k, cc));
          if (c.mode == kModeDev) {
            pub32(k);
          } else {  // the next evaluation is FP64: fold delta into x and publish it
            int64_t gi = base + li;
            for (int cc = 0; cc < D; cc++) {
              A.x[cc * N + gi] += (double)Dl(k, cc);
              Dl(k, cc) = 0.0f;
            }
            publish64(k);
          }
        }
      } else {
        const double cdt = c.dt, keep = c.keep, ratio = c.ratio;
#pragma unroll
        for (int k = 0; k < APT; k++) {
          int li = tid + k * nthr;
          if (li >= cnt) continue;
          int64_t gi = base + li;
          double s[3], mx = 0.0;
#pragma unroll
          for (int cc = 0; cc < D; cc++) {
            double vc = c.reset ? 0.0 : A.v[cc * N + gi];
            const double fk = FD(k, cc);
            vc = fma(keep, fma(cdt, fk, vc), ratio * fk);
            A.v[cc * N + gi] = vc;
            s[cc] = cdt * vc;
            mx = fmax(mx, fabs(s[cc]));
          }
          double scale = 1.0;
          if (mx > 0.5 * fp.max_step) {
            double l2 = 0.0;
#pragma unroll
            for (int cc = 0; cc < D; cc++) l2 += (s[cc] / mx) * (s[cc] / mx);
            double len = mx * sqrt(l2);
            if (len > fp.max_step) scale = fp.max_step / len;
          }
#pragma unroll
          for (int cc = 0; cc < D; cc++) A.x[cc * N + gi] = fma(scale, s[cc], A.x[cc * N + gi]);
          publish64(k);
        }
      }
    } else if (MIXED && c.mode == kModeEval64) {
      // no move: fold delta into the reference and publish FP64 positions
#pragma unroll
      for (int k = 0; k < APT; k++) {
        int li = tid + k * nthr;
        if (li >= cnt) continue;
        int64_t gi = base + li;
        for (int cc = 0; cc < D; cc++) {
          A.x[cc * N + gi] += (double)Dl(k, cc);
          Dl(k, cc) = 0.0f;
        }
        publish64(k);
      }
    }
      csync();  // (B) new positions visible; partial slots free again
    }
    // materialise x = x_ref + delta (mixed)
    if (MIXED) {
#pragma unroll
      for (int k = 0; k < APT; k++) {
        int li = tid + k * nthr;
        if (li >= cnt) continue;
        int64_t gi = base + li;
        for (int c = 0; c < D; c++) {
          A.x[c * N + gi] += (double)Dl(k, c);
          Dl(k, c) = 0.0f;
        }
      }
    }
    if (status == kStatusRebuild && A.inkernel_rebuild) {
      // rebuild the lists here and resume the same FIRE state
      if (rebuild_lists()) {
        kreb++;
        tilt_b = H[1];
#pragma unroll
        for (int k = 0; k < 9; k++) Hb[k] = H[k];
        wmaxf = 0.0f;
        status = kStatusRunning;
        continue;  // republishes FP64 positions; the next evaluation is FP64
      }
    }
    if (status != AQS_OK) break;  // rebuild, budget or error: the next launch resumes
    // ---- step converged: non-affine displacement D_k, records, snapshot ----
    {
      // displacement from the start of the minimisation (d) and from the plain
      // affine start (d + dgamma u when a learned start was used)
      const bool warm = A.warm_u && !(step == 0 && first_noaffine);
      double sv[4] = {0.0, 0.0, 0.0, 0.0}, sa[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < APT; k++) {
        int li = tid + k * nthr;
        if (li >= cnt) continue;
        int64_t gi = base + li;
        double d[3];
        for (int c = 0; c < D; c++) d[c] = A.x[c * N + gi] - A.xs[c * N + gi];
        min_image<D>(H, d);
        for (int c = 0; c < D; c++) sv[c] += d[c];
        if (warm) {
          const float* u = A.warm_u + (g.off + A.perm[gi]) * D;
          for (int c = 0; c < D; c++) sa[c] += d[c] + dgam * (double)u[c];
        }
      }
      cluster_reduce(sv, D, false);
      if (warm) cluster_reduce(sa, D, false);
      double mx[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < APT; k++) {
        int li = tid + k * nthr;
        if (li >= cnt) continue;
        int64_t gi = base + li;
        double d[3], s2 = 0.0, a2 = 0.0;
        for (int c = 0; c < D; c++) d[c] = A.x[c * N + gi] - A.xs[c * N + gi];
        min_image<D>(H, d);
        const float* u = warm ? A.warm_u + (g.off + A.perm[gi]) * D : nullptr;
        for (int c = 0; c < D; c++) {
          double e = d[c] - sv[c] / n;
          s2 += e * e;
          double f = warm ? d[c] + dgam * (double)u[c] - sa[c] / n : e;
          a2 += f * f;
        }
        mx[0] = fmax(mx[0], a2);
        mx[1] = fmax(mx[1], s2);
      }
      cluster_reduce(mx, 2, true);
      if (rank == 0 && tid == 0 && A.rec) {
        double* rec = A.rec + ((int64_t)ri * A.rec_stride + step) * kRecFields;
        rec[0] = E;
        rec[1] = W;
        rec[2] = sqrt(mx[0]);
        rec[3] = (double)iters;
        rec[4] = (double)evals;
        rec[5] = sqrt(mx[1]);
      }
      if (step == 0 && first_noaffine && want_snap && A.snap) {
        double* sp = A.snap + (int64_t)ri * A.snap_stride;
#pragma unroll
        for (int k = 0; k < APT; k++) {
          int li = tid + k * nthr;
          if (li >= cnt) continue;
          int64_t gi = base + li;
          const int u = A.perm[gi];
          for (int c = 0; c < D; c++) sp[(int64_t)u * D + c] = A.x[c * N + gi];
        }
      }
    }
    step++;
    phase = 0;
    status = kStatusRunning;
    if (step >= nsteps) {
      status = AQS_OK;
      break;
    }
    if (launch_iters >= A.launch_budget) break;  // yield; the next launch starts the step
    csync();  // everybody is done with this step before the next one publishes
  }

  // ---- exit: keep v for a resumed minimisation, store the job state ----
  if (MIXED && phase == 1 && !v64) {
#pragma unroll
    for (int k = 0; k < APT; k++) {
      int li = tid + k * nthr;
      if (li >= cnt) continue;
      int64_t gi = base + li;
      for (int c = 0; c < D; c++) A.v[c * N + gi] = (double)V(k, c);
    }
  }
  if (rank == 0 && tid == 0) {
    st->dt = MIXED ? (double)dtf : dt;
    st->alpha = MIXED ? (double)alphaf : alpha;
    st->npos = npos;
    st->iters = iters;
    st->evals64 = evals;
    st->evals32 = evals32;
    st->acc_iters = acc_it;
    st->acc64 = acc64;
    st->acc32 = acc32;
    st->kreb = kreb;
    st->status = status;
    st->fmax = fmx;
    st->step = step;
    st->phase = phase;
    st->tilt = H[1];
    st->tilt_b = tilt_b;
    if (HIST)
      for (int k = 0; k < 9; k++) {
        st->Hc[k] = H[k];
        st->Hb[k] = Hb[k];
      }
    if (status == AQS_OK) {
      st->E = E;
      st->tau = W;
    }
  }
  csync();  // nobody leaves while others may still read its shared memory
}

}  // namespace aqs

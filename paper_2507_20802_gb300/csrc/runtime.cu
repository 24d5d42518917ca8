// runtime.cu -- host runtime and C ABI (include/aqs.h): system state on the
// device, list rebuilds, the batched minimiser driver, sequential AQS and the
// two-level parallel stepping of Sec. 3 (Algorithm 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <functional>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "aqs_internal.cuh"
#include "launch.cuh"
#include "lists.cuh"
#include "minimize.cuh"
#include "misc.cuh"
#include "warm.cuh"

namespace aqs {
static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 1;
  }
  return n;
}
static thread_local std::string g_err;
static std::atomic<int> g_timing{0};
static aqs_kernel_stats g_stats{};

static aqs_status fail(aqs_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}
}  // namespace aqs

using namespace aqs;

#define CUDA_TRY(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(AQS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define AQS_TRY(call)                      \
  do {                                     \
    aqs_status s_ = (call);                \
    if (s_ != AQS_OK) return s_;           \
  } while (0)

struct Alloc {
  void* p;
  size_t bytes;
};

struct aqs_system {
  int dim = 2, R = 0, nt = 0, prec = 0, cap = 0, C_override = 0;
  // cluster-size autotuner: iterations per candidate (0 = off) and the
  // choices made so far, keyed by (replicas in flight, largest N)
  int64_t tune_iters = 0;
  bool tuning = false;
  struct Tuned {
    int C, staging, tpa;
    bool gb;
  };
  std::map<std::pair<int, int64_t>, Tuned> tuned;
  // threads per atom of the force phase (1 or 2; the autotuner may choose 2
  // where 2 npc threads fit a CTA); tpa_user marks a caller's choice
  int tpa = 1;
  bool tpa_user = false;
  // grid barriers (aqs_set_grid_barrier): the replicas' CTAs run in one
  // cooperative launch without clusters and synchronise through global memory
  bool grid_barrier = false;
  bool grid_barrier_user = false;
  double* gb_part = nullptr;
  unsigned* gb_bar = nullptr;  // one 64-bit arrival counter per replica
  int* gb_err = nullptr;
  // staging mode of the minimiser launches (-1: automatic); staging_user marks
  // a mode the caller fixed, which the tuner leaves alone
  int staging = -1;
  bool staging_user = false;
  // FIRE iterations a replica runs per persistent launch before the host
  // regroups the replicas still running (larger clusters, stopped chains)
  int64_t launch_budget = 2048;
  aqs_potential pot{};
  double skin = 0.3, rcmax = 0.0, rlist = 0.0;
  cudaStream_t stream = nullptr;
  void* (*ualloc)(size_t, void*) = nullptr;
  void (*ufree)(void*, void*) = nullptr;
  void* actx = nullptr;
  std::vector<int64_t> n, off;
  int64_t ntot = 0, nmax = 0;
  std::vector<RepGeom> geom;
  std::vector<RepState> st;
  std::vector<double> mean_nb;
  std::vector<int64_t> nnb_sum;
  int64_t* d_nnbsum = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // launches of different cluster sizes run concurrently on these streams
  cudaStream_t aux[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t aux_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  PairCoef coef[AQS_MAX_TYPES * AQS_MAX_TYPES];
  float rl2f[AQS_MAX_TYPES * AQS_MAX_TYPES];
  int total_cells = 0, cells_cap = 0;
  std::vector<Alloc> allocs;
  // device arrays
  RepGeom* d_geom = nullptr;
  RepState* d_state = nullptr;
  PairCoef* d_coef = nullptr;
  int* d_work = nullptr;
  uint8_t* d_flag = nullptr;
  int32_t* d_rep_of = nullptr;
  double *x = nullptr, *v = nullptr, *fref = nullptr, *dl = nullptr, *xs = nullptr, *xb = nullptr;
  double *tmp = nullptr, *d_dg = nullptr, *ubuf = nullptr, *ubuf2 = nullptr;
  int32_t *type = nullptr, *perm = nullptr, *inv = nullptr, *cell = nullptr, *key = nullptr;
  int32_t *itmp = nullptr, *nnb = nullptr, *count = nullptr, *cstart = nullptr, *cell_rep = nullptr;
  int32_t* overflow = nullptr;
  int64_t* order = nullptr;
  uint32_t* nb = nullptr;
  size_t nb_bytes = 0;
  CmpJob* d_jobs = nullptr;
  double* d_cmp = nullptr;
  double* d_partial = nullptr;
  int64_t* d_i64 = nullptr;  // small scratch (copy offsets)
  double* d_shift = nullptr;
  double* pubg = nullptr;  // [ntot] position records (16 B in 2D, 32 B in 3D)
  float* lean32 = nullptr;  // per-atom minimiser state of large-CTA launches
  double* lean64 = nullptr;
  // per-step job records and first-step snapshots
  double* d_rec = nullptr;
  int64_t rec_cap = 0;
  double* d_snap = nullptr;
  // learned warm start buffers (allocated on first use)
  __nv_bfloat16* d_feat = nullptr;
  float* d_u = nullptr;
  double* d_save = nullptr;
  int* d_err = nullptr;
  // deformation histories: the rotation Q (row-major d x d) from the stored
  // frame, where every cell is upper triangular, to the laboratory frame
  // (H_lab = Q H); the identity unless a history rotated the cell
  std::vector<std::array<double, 9>> frame;
  double* d_hist = nullptr;  // [R][hist_cap][kHistFields] job map tables
  int64_t hist_cap = 0;
  double* d_maps = nullptr;  // [R][9] one-increment maps (aqs_deform, level I)
  bool hist_launch = false;  // the running job set uses a map table
  // two-level stepping resources
  aqs_system* chains = nullptr;
  double* snap = nullptr;
  double* ends = nullptr;
};

namespace {

void* dalloc(aqs_system* s, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (s->ualloc) {
    p = s->ualloc(bytes, s->actx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p && (reinterpret_cast<uintptr_t>(p) & 15u)) {  // the kernels need 16-byte alignment
    if (s->ufree) s->ufree(p, s->actx);
    return nullptr;
  }
  if (p) s->allocs.push_back({p, bytes});
  return p;
}

void dfree(aqs_system* s, void* p) {
  if (!p) return;
  for (size_t i = 0; i < s->allocs.size(); i++)
    if (s->allocs[i].p == p) {
      if (s->ufree) s->ufree(p, s->actx);
      else cudaFree(p);
      s->allocs.erase(s->allocs.begin() + i);
      return;
    }
}

template <typename T>
aqs_status alloc_arr(aqs_system* s, T** p, size_t count) {
  *p = static_cast<T*>(dalloc(s, count * sizeof(T)));
  if (!*p) return fail(AQS_ERR_OOM, "device allocation of %zu bytes failed", count * sizeof(T));
  return AQS_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

double lj_u(double r, double sig, double eps) {
  double sr = sig / r, sr2 = sr * sr, sr6 = sr2 * sr2 * sr2;
  return 4.0 * eps * (sr6 * sr6 - sr6);
}
double lj_du(double r, double sig, double eps) {
  double sr = sig / r, sr2 = sr * sr, sr6 = sr2 * sr2 * sr2;
  return -24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r;
}

// perpendicular widths of an upper-triangular cell whose only tilt is H[0][1]
void cell_widths(int D, const double* H, double* w) {
  double Ly = H[1 * D + 1], t = H[0 * D + 1];
  w[0] = H[0] / std::sqrt(1.0 + (t / Ly) * (t / Ly));
  w[1] = Ly;
  if (D == 3) w[2] = H[8];
}

// Cluster size for R concurrently minimised replicas of n atoms: the largest
// C (at most 16 and SMs / R, at least 32 atoms and at most 4096 atoms per CTA)
// at which the device holds all R clusters at once (cudaOccupancyMaxActiveClusters;
// clusters are placed per GPC, so e.g. 23 clusters of 6 CTAs fit a GB300 but
// only 15 of 7-9).  When no size holds all R, the size with the most resident
// CTAs.
int auto_cluster(int dim, bool mixed, int R, int64_t n, int nt, int cap) {
  const int Cmax = (int)std::min<int64_t>(
      std::min<int64_t>(kMaxCluster, std::max(1, sm_count() / std::max(1, R))),
      std::max<int64_t>(1, n / 32));
  int fallback = 0, most = -1;
  for (int C = Cmax; C >= 1; C--) {
    const int64_t npc = (n + C - 1) / C;
    if (npc > 4096) break;
    const int m = minimize_max_active_clusters(dim, mixed, C, (int)npc, (int)n, nt, cap);
    if (m >= std::max(1, R)) return C;
    if (m > 0 && (int64_t)m * C > most) {
      most = m * C;
      fallback = C;
    }
  }
  if (fallback > 0) return fallback;
  int C = 1;
  while ((n + C - 1) / C > 4096 && C < kMaxCluster) C++;
  return C;
}

// Grid-barrier launches: the largest C (at most 16, at least 32 atoms and at
// most 4096 atoms per CTA) at which R replicas' CTAs are all resident.
int gb_cluster(int dim, bool mixed, int R, int64_t n, int nt, int cap, int staging) {
  const int Cmax = (int)std::min<int64_t>(kMaxCluster, std::max<int64_t>(1, n / 32));
  for (int C = Cmax; C >= 1; C--) {
    const int64_t npc = (n + C - 1) / C;
    if (npc > 4096) break;
    if (minimize_max_grid_replicas(dim, mixed, C, (int)npc, (int)n, nt, cap, staging) >= R)
      return C;
  }
  return 0;
}

aqs_status upload_geom(aqs_system* s) {
  CUDA_TRY(cudaMemcpyAsync(s->d_geom, s->geom.data(), sizeof(RepGeom) * s->R,
                           cudaMemcpyHostToDevice, s->stream));
  return AQS_OK;
}

aqs_status upload_state(aqs_system* s) {
  CUDA_TRY(cudaMemcpyAsync(s->d_state, s->st.data(), sizeof(RepState) * s->R,
                           cudaMemcpyHostToDevice, s->stream));
  return AQS_OK;
}

aqs_status download_state(aqs_system* s) {
  CUDA_TRY(cudaMemcpyAsync(s->st.data(), s->d_state, sizeof(RepState) * s->R,
                           cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  // the kernels own the tilt while they shear; mirror it into the geometry
  bool changed = false;
  for (int r = 0; r < s->R; r++) {
    if (s->hist_launch) {
      for (int k = 0; k < s->dim * s->dim; k++)
        if (s->geom[r].H[k] != s->st[r].Hc[k]) {
          s->geom[r].H[k] = s->st[r].Hc[k];
          changed = true;
        }
    } else if (s->geom[r].H[1] != s->st[r].tilt) {
      s->geom[r].H[1] = s->st[r].tilt;
      changed = true;
    }
    std::memcpy(s->st[r].Hc, s->geom[r].H, sizeof(s->st[r].Hc));
  }
  if (changed) AQS_TRY(upload_geom(s));
  return AQS_OK;
}

// after the host changed a cell: the kernel-side copy of the tilt follows
void sync_tilt_to_state(aqs_system* s) {
  for (int r = 0; r < s->R; r++) {
    s->st[r].tilt = s->geom[r].H[1];
    std::memcpy(s->st[r].Hc, s->geom[r].H, sizeof(s->st[r].Hc));
  }
}

BuildArgs build_args(aqs_system* s) {
  BuildArgs a;
  a.geom = s->d_geom;
  a.rep_of = s->d_rep_of;
  a.flag = s->d_flag;
  a.x = s->x;
  a.v = s->v;
  a.xs = s->xs;
  a.xb = s->xb;
  a.type = s->type;
  a.perm = s->perm;
  a.inv = s->inv;
  a.cell = s->cell;
  a.key = s->key;
  a.order = s->order;
  a.count = s->count;
  a.cstart = s->cstart;
  a.cell_rep = s->cell_rep;
  a.tmp = s->tmp;
  a.itmp = s->itmp;
  a.nb = s->nb;
  a.nnb = s->nnb;
  a.overflow = s->overflow;
  for (int k = 0; k < AQS_MAX_TYPES * AQS_MAX_TYPES; k++) a.rl2f[k] = s->rl2f[k];
  a.nt = s->nt;
  a.cap = s->cap;
  a.ntot = s->ntot;
  return a;
}

aqs_status layout_lists(aqs_system* s) {
  int64_t total = 0;
  for (int r = 0; r < s->R; r++) {
    s->geom[r].nb_off = total;
    total += (int64_t)s->cap * s->n[r];
  }
  if (s->nb) dfree(s, s->nb);
  s->nb = nullptr;
  s->nb_bytes = sizeof(uint32_t) * (size_t)total;
  return alloc_arr(s, &s->nb, (size_t)total);
}

// Rebuild cells and Verlet lists of the replicas with flags[r] != 0.
aqs_status rebuild(aqs_system* s, const std::vector<uint8_t>& flags, int depth = 0) {
  const int D = s->dim;
  bool any = false;
  for (int r = 0; r < s->R; r++) {
    if (!flags[r]) continue;
    any = true;
    double w[3];
    cell_widths(D, s->geom[r].H, w);
    int ncell = 1;
    for (int c = 0; c < D; c++) {
      int k = (int)std::floor(w[c] / s->rlist);
      if (k < 3)
        return fail(AQS_ERR_BOX_TOO_SMALL,
                    "replica %d: perpendicular cell width %.4g below 3 (rc+skin) = %.4g", r, w[c],
                    3 * s->rlist);
      k = std::min(k, 1024);
      s->geom[r].nc[c] = k;
      ncell *= k;
    }
    if (D == 2) s->geom[r].nc[2] = 1;
    s->geom[r].ncell = ncell;
  }
  if (!any) return AQS_OK;
  int total = 0;
  std::vector<int32_t> cell_rep;
  for (int r = 0; r < s->R; r++) {
    s->geom[r].cell_off = total;
    total += s->geom[r].ncell + 1;
  }
  cell_rep.resize(total);
  for (int r = 0; r < s->R; r++)
    for (int c = 0; c <= s->geom[r].ncell; c++) cell_rep[s->geom[r].cell_off + c] = r;
  if (total > s->cells_cap) {
    dfree(s, s->count);
    dfree(s, s->cstart);
    dfree(s, s->cell_rep);
    s->cells_cap = std::max(total, 2 * s->cells_cap);
    AQS_TRY(alloc_arr(s, &s->count, s->cells_cap));
    AQS_TRY(alloc_arr(s, &s->cstart, s->cells_cap));
    AQS_TRY(alloc_arr(s, &s->cell_rep, s->cells_cap));
  }
  s->total_cells = total;
  CUDA_TRY(cudaMemcpyAsync(s->cell_rep, cell_rep.data(), sizeof(int32_t) * total,
                           cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(cudaMemcpyAsync(s->d_flag, flags.data(), s->R, cudaMemcpyHostToDevice, s->stream));
  AQS_TRY(upload_geom(s));
  {
    BuildArgs a = build_args(s);
    CUDA_TRY(cudaMemsetAsync(s->count, 0, sizeof(int32_t) * total, s->stream));
    CUDA_TRY(cudaMemsetAsync(s->overflow, 0, sizeof(int32_t) * s->R, s->stream));
    CUDA_TRY(launch_rebuild_bin(D, a, s->R, s->stream));
    CUDA_TRY(launch_rebuild_sort(D, a, total, s->stream));
    CUDA_TRY(launch_rebuild_verlet(D, a, s->stream));
    CUDA_TRY(launch_sum_nnb(a, s->R, s->d_nnbsum, s->stream));
    std::vector<int32_t> over(s->R);
    std::vector<int64_t> sums(s->R);
    CUDA_TRY(cudaMemcpyAsync(over.data(), s->overflow, sizeof(int32_t) * s->R,
                             cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaMemcpyAsync(sums.data(), s->d_nnbsum, sizeof(int64_t) * s->R,
                             cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    for (int r = 0; r < s->R; r++)
      if (flags[r]) s->nnb_sum[r] = sums[r];
    int need = 0;
    for (int r = 0; r < s->R; r++) need = std::max(need, over[r]);
    if (need > 0) {
      // grow the list; every replica's block moves, so all of them are rebuilt
      if (depth >= 6) return fail(AQS_ERR_NLIST_OVERFLOW, "neighbour list keeps overflowing");
      s->cap = std::max((int)(s->cap * 1.5), need + 16);
      AQS_TRY(layout_lists(s));
      return rebuild(s, std::vector<uint8_t>(s->R, 1), depth + 1);
    }
  }
  for (int r = 0; r < s->R; r++)
    if (flags[r]) {
      s->geom[r].tilt_b = s->geom[r].H[0 * D + 1];
      s->st[r].tilt_b = s->geom[r].tilt_b;
      s->st[r].tilt = s->geom[r].H[0 * D + 1];
      std::memcpy(s->st[r].Hb, s->geom[r].H, sizeof(s->st[r].Hb));
      std::memcpy(s->st[r].Hc, s->geom[r].H, sizeof(s->st[r].Hc));
    }
  AQS_TRY(upload_geom(s));
  AQS_TRY(upload_state(s));
  return AQS_OK;
}

aqs_status rebuild_all(aqs_system* s) { return rebuild(s, std::vector<uint8_t>(s->R, 1)); }

void make_coef(aqs_system* s, const aqs_potential& p) {
  s->rcmax = 0.0;
  for (int a = 0; a < s->nt; a++)
    for (int b = 0; b < s->nt; b++) {
      int k = a * s->nt + b;
      double sig = p.sigma[a * s->nt + b], eps = p.eps[a * s->nt + b];
      double rc = p.rc_factor * sig;
      PairCoef& c = s->coef[k];
      double s6 = std::pow(sig, 6.0);
      c.A = -48.0 * eps * s6 * s6;
      c.B = 24.0 * eps * s6;
      c.C = -lj_du(rc, sig, eps);
      c.rc = rc;
      c.rc2 = rc * rc;
      c.rl2 = (rc + s->skin) * (rc + s->skin);
      c.e12 = 4.0 * eps * s6 * s6;
      c.e6 = 4.0 * eps * s6;
      c.Uc = lj_u(rc, sig, eps);
      c.dUc = lj_du(rc, sig, eps);
      c.Af = (float)c.A;
      c.Bf = (float)c.B;
      c.Cf = (float)c.C;
      c.rc2f = (float)c.rc2;
      double rl = (rc + s->skin) * (1.0 + 1e-6) + 1e-6;  // FP32 rounding margin
      s->rl2f[k] = (float)(rl * rl);
      s->rcmax = std::max(s->rcmax, rc);
    }
  s->rlist = s->rcmax + s->skin;
}

FireDev fire_dev(const aqs_fire_params* f) {
  FireDev d;
  d.dt0 = f->dt0;
  d.alpha0 = f->alpha0;
  d.f_inc = f->f_inc;
  d.f_dec = f->f_dec;
  d.f_alpha = f->f_alpha;
  d.dt_max = f->dt_max;
  d.dt_min = f->dt_min;
  d.max_step = f->max_step;
  d.tol = f->tol;
  d.ref_ratio = f->ref_ratio;
  d.ref_dmax = f->ref_dmax;
  d.n_min = f->n_min;
  d.max_iter = f->max_iter;
  return d;
}

MinArgs min_args(aqs_system* s, const aqs_fire_params* f) {
  MinArgs a;
  a.geom = s->d_geom;
  a.state = s->d_state;
  a.work = s->d_work;
  a.x = s->x;
  a.v = s->v;
  a.fref = s->fref;
  a.dl = s->dl;
  a.xs = s->xs;
  a.xb = s->xb;
  a.type = s->type;
  a.cell = s->cell;
  a.nb = s->nb;
  a.nnb = s->nnb;
  a.coef = s->d_coef;
  a.ntot = s->ntot;
  a.nt = s->nt;
  a.fire = fire_dev(f);
  a.skin = s->skin;
  a.rlist = s->rlist;
  a.launch_budget = s->launch_budget;
  a.npc_launch = 0;
  a.nrep_launch = 0;
  a.rec = s->d_rec;
  a.rec_stride = s->rec_cap;
  a.snap = s->d_snap;
  a.snap_stride = (int64_t)s->dim * s->nmax;
  a.perm = s->perm;
  a.warm_u = nullptr;
  a.count = s->count;
  a.cstart = s->cstart;
  a.cellatoms = s->itmp;  // host rebuilds use it only between launches
  a.cap = s->cap;
  a.inkernel_rebuild = 1;
  a.pubg = s->pubg;
  a.lean32 = s->lean32;
  a.lean64 = s->lean64;
  a.hist = nullptr;
  a.hist_stride = 0;
  a.gb_C = 0;
  a.gb_part = nullptr;
  a.gb_bar = nullptr;
  a.gb_err = nullptr;
  for (int k = 0; k < AQS_MAX_TYPES * AQS_MAX_TYPES; k++) a.rl2f[k] = s->rl2f[k];
  return a;
}

// Per-replica job: nsteps fine steps of increment dgamma (affine map, then
// FIRE to convergence); first_noaffine skips the map of the first step and
// want_snap stores the caller-order positions after that first step.
struct Job {
  int64_t nsteps = 0;
  double dgamma = 0.0;
  int first_noaffine = 0;
  int want_snap = 0;
  // deformation history: nsteps x kHistFields rows (map, new cell) per job
  // step; empty = simple shear by dgamma
  std::vector<double> table;
};

struct JobOut {
  std::vector<double> rec;  // [R][nsteps_max][kRecFields]
  int64_t stride = 0;
  std::vector<int64_t> rebuilds;
};

aqs_status ensure_records(aqs_system* s, int64_t nsteps, bool snap) {
  if (nsteps > s->rec_cap) {
    dfree(s, s->d_rec);
    s->rec_cap = std::max<int64_t>(nsteps, 2 * s->rec_cap);
    AQS_TRY(alloc_arr(s, &s->d_rec, (size_t)s->R * s->rec_cap * kRecFields));
  }
  if (snap && !s->d_snap) AQS_TRY(alloc_arr(s, &s->d_snap, (size_t)s->R * s->dim * s->nmax));
  return AQS_OK;
}

aqs_status tune_clusters(aqs_system* s, const aqs_fire_params* f, const std::vector<uint8_t>& mask,
                         int64_t iters, int* best, int* best_staging, double* ms_per_iter,
                         double* ms_per_staging);
aqs_status apply_cluster(aqs_system* s, const std::vector<int>& reps, int C);

// Called by run_jobs after every pass with the replicas that are still
// running; it may remove replicas whose results are no longer needed (they
// are marked in `dropped` and stop without a final status).
using PassHook = std::function<aqs_status(std::vector<int>& next, std::vector<uint8_t>& dropped)>;

// Runs the jobs of the replicas with jobs[r].nsteps > 0 to completion in
// persistent launches (one per cluster size and pass); between passes only
// list rebuilds and budget yields are handled on the host.
aqs_status run_jobs(aqs_system* s, const aqs_fire_params* f, const std::vector<Job>& jobs,
                    JobOut* out, const float* warm_u = nullptr, const PassHook* hook = nullptr,
                    std::vector<uint8_t>* dropped_out = nullptr) {
  std::vector<uint8_t> dropped(s->R, 0);
  if (s->tune_iters > 0 && s->C_override <= 0 && !s->tuning) {
    std::vector<uint8_t> mask(s->R, 0);
    std::vector<int> reps;
    int64_t nmax = 0;
    for (int r = 0; r < s->R; r++)
      if (jobs[r].nsteps > 0) {
        mask[r] = 1;
        reps.push_back(r);
        nmax = std::max(nmax, s->n[r]);
      }
    if (!reps.empty()) {
      const auto key = std::make_pair((int)reps.size(), nmax);
      auto it = s->tuned.find(key);
      if (it == s->tuned.end()) {
        int best = 0, mode = -1;
        AQS_TRY(tune_clusters(s, f, mask, s->tune_iters, &best, &mode, nullptr, nullptr));
        s->tuned[key] = aqs_system::Tuned{best, mode, s->tpa, s->grid_barrier};
      } else {
        if (!s->staging_user) s->staging = it->second.staging;
        if (!s->tpa_user) s->tpa = it->second.tpa;
        if (!s->grid_barrier_user) s->grid_barrier = it->second.gb;
        AQS_TRY(apply_cluster(s, reps, it->second.C));
      }
    }
  }
  if (s->grid_barrier && s->C_override <= 0 && !s->tuning && s->tune_iters <= 0) {
    // one cooperative launch holds every replica: one C for all of them
    std::vector<int> reps;
    int64_t nmax = 0;
    for (int r = 0; r < s->R; r++)
      if (jobs[r].nsteps > 0) {
        reps.push_back(r);
        nmax = std::max(nmax, s->n[r]);
      }
    if (!reps.empty()) {
      const int C = gb_cluster(s->dim, s->prec == AQS_MIXED, (int)reps.size(), nmax, s->nt,
                               s->cap, s->staging);
      if (C <= 0) return fail(AQS_ERR_UNSUPPORTED, "grid barriers: the replicas do not fit the device");
      AQS_TRY(apply_cluster(s, reps, C));
    }
  }
  if (s->grid_barrier && !s->gb_part) {
    AQS_TRY(alloc_arr(s, &s->gb_part, (size_t)s->R * kMaxCluster * kNumRed));
    AQS_TRY(alloc_arr(s, &s->gb_bar, (size_t)2 * s->R));
    AQS_TRY(alloc_arr(s, &s->gb_err, (size_t)1));
    CUDA_TRY(cudaMemsetAsync(s->gb_bar, 0, sizeof(unsigned) * 2 * s->R, s->stream));
    CUDA_TRY(cudaMemsetAsync(s->gb_err, 0, sizeof(int), s->stream));
  }
  int64_t maxsteps = 0;
  bool snap = false;
  std::vector<int> todo;
  for (int r = 0; r < s->R; r++)
    if (jobs[r].nsteps > 0) {
      todo.push_back(r);
      maxsteps = std::max(maxsteps, jobs[r].nsteps);
      snap = snap || jobs[r].want_snap;
      RepState& t = s->st[r];
      t.nsteps = jobs[r].nsteps;
      t.dgamma = jobs[r].dgamma;
      t.first_noaffine = jobs[r].first_noaffine;
      t.want_snap = jobs[r].want_snap;
      t.step = 0;
      t.phase = 0;
      t.status = kStatusRunning;
      t.tilt = s->geom[r].H[1];
    }
  if (todo.empty()) return AQS_OK;
  AQS_TRY(ensure_records(s, maxsteps, snap));
  // deformation histories: every job of the set gets a table (jobs without
  // one get the rows of their simple shear), uploaded [R][maxsteps][18]
  bool any_table = false;
  for (int r : todo) any_table = any_table || !jobs[r].table.empty();
  s->hist_launch = any_table;
  if (any_table) {
    if (maxsteps > s->hist_cap) {
      dfree(s, s->d_hist);
      s->hist_cap = std::max<int64_t>(maxsteps, 2 * s->hist_cap);
      AQS_TRY(alloc_arr(s, &s->d_hist, (size_t)s->R * s->hist_cap * kHistFields));
    }
    std::vector<double> all((size_t)s->R * s->hist_cap * kHistFields, 0.0);
    for (int r : todo) {
      double* dst = all.data() + (size_t)r * s->hist_cap * kHistFields;
      if (!jobs[r].table.empty()) {
        std::copy(jobs[r].table.begin(), jobs[r].table.end(), dst);
        continue;
      }
      double H[9];
      std::memcpy(H, s->geom[r].H, sizeof(H));
      for (int64_t k = 0; k < jobs[r].nsteps; k++) {
        double* row = dst + k * kHistFields;
        for (int a = 0; a < 3; a++) row[a * 3 + a] = 1.0;
        if (!(k == 0 && jobs[r].first_noaffine)) {
          row[1] = jobs[r].dgamma;
          H[1] = std::fma(jobs[r].dgamma, H[s->dim + 1], H[1]);
        }
        for (int a = 0; a < s->dim; a++)
          for (int c = 0; c < s->dim; c++) row[9 + a * 3 + c] = H[a * s->dim + c];
      }
    }
    CUDA_TRY(cudaMemcpyAsync(s->d_hist, all.data(), sizeof(double) * all.size(),
                             cudaMemcpyHostToDevice, s->stream));
    for (int r : todo) {
      std::memcpy(s->st[r].Hc, s->geom[r].H, sizeof(s->st[r].Hc));
      // a simple-shear launch may have rebuilt the list in the kernel since
      // Hb was written; only the tilt changes there
      s->st[r].Hb[1] = s->st[r].tilt_b;
    }
  }
  AQS_TRY(upload_state(s));
  std::vector<int64_t> rebuilds(s->R, 0);
  std::vector<int> kreb0(s->R);
  for (int r = 0; r < s->R; r++) kreb0[r] = s->st[r].kreb;
  std::vector<int> order_work;
  for (int64_t pass = 0; pass < 100000000 && !todo.empty(); pass++) {
    std::vector<int> Cs;
    for (int r : todo) Cs.push_back(s->geom[r].C);
    std::sort(Cs.begin(), Cs.end());
    Cs.erase(std::unique(Cs.begin(), Cs.end()), Cs.end());
    order_work.clear();
    std::vector<std::pair<int, int>> groups;
    for (int C : Cs) {
      int start = (int)order_work.size();
      for (int r : todo)
        if (s->geom[r].C == C) order_work.push_back(r);
      groups.push_back({start, (int)order_work.size() - start});
    }
    if (s->grid_barrier && groups.size() > 1)
      return fail(AQS_ERR_UNSUPPORTED, "grid barriers need one cluster size for all replicas");
    CUDA_TRY(cudaMemcpyAsync(s->d_work, order_work.data(), sizeof(int) * order_work.size(),
                             cudaMemcpyHostToDevice, s->stream));
    if (!s->lean32) {  // first lean launch of this system
      bool lean = false;
      for (int r : todo) lean = lean || minimize_launch_is_lean(s->dim, s->geom[r].npc, s->tpa);
      if (lean) {
        AQS_TRY(alloc_arr(s, &s->lean32, (size_t)15 * s->ntot));
        AQS_TRY(alloc_arr(s, &s->lean64, (size_t)3 * s->ntot));
      }
    }
    MinArgs a = min_args(s, f);
    a.warm_u = warm_u;
    if (s->grid_barrier) {
      a.gb_part = s->gb_part;
      a.gb_bar = s->gb_bar;
      a.gb_err = s->gb_err;
    }
    if (s->hist_launch) {
      a.hist = s->d_hist;
      a.hist_stride = s->hist_cap;
    }
    const bool timing = g_timing.load() != 0;
    std::vector<RepState> before(s->st);
    if (timing) CUDA_TRY(cudaEventRecord(s->ev0, s->stream));
    const bool multi = groups.size() > 1;
    if (multi) {
      if (!s->aux[0])
        for (int k = 0; k < 4; k++) {
          CUDA_TRY(cudaStreamCreateWithFlags(&s->aux[k], cudaStreamNonBlocking));
          CUDA_TRY(cudaEventCreateWithFlags(&s->aux_ev[k], cudaEventDisableTiming));
        }
      if (!s->aux_ev[4]) CUDA_TRY(cudaEventCreateWithFlags(&s->aux_ev[4], cudaEventDisableTiming));
      CUDA_TRY(cudaEventRecord(s->aux_ev[4], s->stream));
    }
    for (size_t gi = 0; gi < groups.size(); gi++) {
      int C = Cs[gi];
      int npc = 0, nrep = 0;
      for (int k = 0; k < groups[gi].second; k++) {
        npc = std::max(npc, s->geom[order_work[groups[gi].first + k]].npc);
        nrep = std::max(nrep, s->geom[order_work[groups[gi].first + k]].n);
      }
      a.work = s->d_work + groups[gi].first;
      cudaStream_t st = s->stream;
      if (multi) {
        st = s->aux[gi % 4];
        CUDA_TRY(cudaStreamWaitEvent(st, s->aux_ev[4], 0));
      }
      if (s->grid_barrier)  // the barrier counters start at zero in every launch
        CUDA_TRY(cudaMemsetAsync(s->gb_bar, 0, sizeof(unsigned) * 2 * s->R, st));
      CUDA_TRY(launch_minimize(s->dim, s->prec == AQS_MIXED, a, groups[gi].second, C, npc, nrep,
                               s->cap, st, s->staging, s->tpa, s->grid_barrier));
      if (multi) CUDA_TRY(cudaEventRecord(s->aux_ev[gi % 4], st));
      if (multi && (gi % 4 == 3 || gi + 1 == groups.size()))
        for (size_t k = 0; k <= gi % 4; k++) CUDA_TRY(cudaStreamWaitEvent(s->stream, s->aux_ev[k], 0));
    }
    if (timing) CUDA_TRY(cudaEventRecord(s->ev1, s->stream));
    AQS_TRY(download_state(s));
    if (s->grid_barrier) {
      int err = 0;
      CUDA_TRY(cudaMemcpy(&err, s->gb_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (err) {
        // the barrier words may be left mid-barrier: clear them for the next call
        CUDA_TRY(cudaMemsetAsync(s->gb_bar, 0, sizeof(unsigned) * 2 * s->R, s->stream));
        CUDA_TRY(cudaMemsetAsync(s->gb_err, 0, sizeof(int), s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        return fail(AQS_ERR_TIMEOUT, "a grid-barrier wait ran out (CTAs not resident?)");
      }
    }
    if (timing) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
      g_stats.launches += (int64_t)groups.size();
      g_stats.kernel_ms += ms;
      for (int r : todo) {
        int64_t d32 = s->st[r].acc32 - before[r].acc32;
        int64_t d64 = s->st[r].acc64 - before[r].acc64;
        int64_t dit = s->st[r].acc_iters - before[r].acc_iters;
        g_stats.evals32 += d32;
        g_stats.evals64 += d64;
        g_stats.pairs32 += d32 * s->nnb_sum[r];
        g_stats.pairs64 += d64 * s->nnb_sum[r];
        g_stats.atom_iters += dit * s->n[r];
        g_stats.rebuilds += s->st[r].kreb - before[r].kreb;
      }
    }
    std::vector<uint8_t> flags(s->R, 0);
    std::vector<int> next;
    for (int r : todo) {
      const int st = s->st[r].status;
      if (st == kStatusRebuild) {
        flags[r] = 1;
        rebuilds[r]++;
      }
      if (st == kStatusRebuild || st == kStatusRunning) next.push_back(r);
    }
    if (hook && !next.empty()) {
      AQS_TRY((*hook)(next, dropped));
      for (int r = 0; r < s->R; r++)
        if (dropped[r]) flags[r] = 0;
    }
    // fewer replicas left: give each a larger cluster (the list is rebuilt
    // for the new owner layout; the FIRE state carries over)
    if (s->C_override <= 0 && !next.empty() && next.size() < todo.size()) {
      int Cg = 0;
      if (s->grid_barrier) {
        int64_t nmax = 0;
        for (int r : next) nmax = std::max(nmax, s->n[r]);
        Cg = gb_cluster(s->dim, s->prec == AQS_MIXED, (int)next.size(), nmax, s->nt, s->cap,
                        s->staging);
      }
      for (int r : next) {
        int Cn = s->grid_barrier ? Cg
                                 : auto_cluster(s->dim, s->prec == AQS_MIXED, (int)next.size(),
                                                s->n[r], s->nt, s->cap);
        if (Cn > s->geom[r].C) {
          s->geom[r].C = Cn;
          s->geom[r].npc = (int)((s->n[r] + Cn - 1) / Cn);
          flags[r] = 1;
        }
      }
    }
    if (!next.empty() && std::count(flags.begin(), flags.end(), 1) > 0) AQS_TRY(rebuild(s, flags));
    todo.swap(next);
  }
  s->hist_launch = false;
  if (!todo.empty()) return fail(AQS_ERR_TIMEOUT, "minimiser jobs did not finish");
  if (out) {
    out->stride = s->rec_cap;
    out->rec.assign((size_t)s->R * s->rec_cap * kRecFields, 0.0);
    CUDA_TRY(cudaMemcpyAsync(out->rec.data(), s->d_rec, sizeof(double) * out->rec.size(),
                             cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    out->rebuilds = rebuilds;
    for (int r = 0; r < s->R; r++) out->rebuilds[r] += s->st[r].kreb - kreb0[r];
  }
  aqs_status first = AQS_OK;
  if (dropped_out) *dropped_out = dropped;
  for (int r = 0; r < s->R; r++) {
    if (jobs[r].nsteps <= 0 || dropped[r]) continue;
    const RepState& t = s->st[r];
    if (t.status != AQS_OK && first == AQS_OK) {
      first = (aqs_status)t.status;
      fail(first, "replica %d: minimiser status %d at step %lld after %lld iterations (fmax %.3g)",
           r, t.status, (long long)t.step, (long long)t.iters, t.fmax);
    }
  }
  return first;
}

// One minimisation (a one-step job without affine map) of the masked replicas.
aqs_status minimize_impl(aqs_system* s, const aqs_fire_params* f, const std::vector<uint8_t>& mask,
                         aqs_min_result* res) {
  std::vector<Job> jobs(s->R);
  for (int r = 0; r < s->R; r++)
    if (mask[r]) {
      jobs[r].nsteps = 1;
      jobs[r].first_noaffine = 1;
    }
  JobOut out;
  aqs_status st = run_jobs(s, f, jobs, &out);
  for (int r = 0; r < s->R; r++) {
    if (!mask[r] || !res) continue;
    const RepState& t = s->st[r];
    const double* rec = &out.rec[(size_t)r * out.stride * kRecFields];
    aqs_min_result& o = res[r];
    o.iters = t.status == AQS_OK ? (int64_t)rec[3] : t.iters;
    o.evals64 = t.status == AQS_OK ? (int64_t)rec[4] : t.evals64;
    o.rebuilds = out.rebuilds.empty() ? 0 : out.rebuilds[r];
    o.energy = t.status == AQS_OK ? rec[0] : 0.0;
    o.fmax = t.fmax;
    o.tau = t.status == AQS_OK ? rec[1] : 0.0;
    o.nonaffine = t.status == AQS_OK ? rec[2] : 0.0;
    o.status = t.status;
  }
  return st;
}

aqs_status affine_impl(aqs_system* s, const std::vector<double>& dg) {
  const int D = s->dim;
  bool any = false;
  for (int r = 0; r < s->R; r++) {
    if (dg[r] == 0.0) continue;
    any = true;
    s->geom[r].H[0 * D + 1] += dg[r] * s->geom[r].H[1 * D + 1];
  }
  if (!any) return AQS_OK;
  AQS_TRY(upload_geom(s));
  sync_tilt_to_state(s);
  AQS_TRY(upload_state(s));
  CUDA_TRY(cudaMemcpyAsync(s->d_dg, dg.data(), sizeof(double) * s->R, cudaMemcpyHostToDevice,
                           s->stream));
  CUDA_TRY(launch_affine(s->x, s->xb, s->d_rep_of, s->d_dg, s->ntot, s->stream));
  return AQS_OK;
}

aqs_status alloc_system(aqs_system* s) {
  const int D = s->dim;
  const int64_t N = s->ntot;
  AQS_TRY(alloc_arr(s, &s->d_geom, s->R));
  AQS_TRY(alloc_arr(s, &s->d_state, s->R));
  AQS_TRY(alloc_arr(s, &s->d_coef, AQS_MAX_TYPES * AQS_MAX_TYPES));
  AQS_TRY(alloc_arr(s, &s->d_work, s->R));
  AQS_TRY(alloc_arr(s, &s->d_flag, s->R));
  AQS_TRY(alloc_arr(s, &s->d_rep_of, N));
  AQS_TRY(alloc_arr(s, &s->x, D * N));
  AQS_TRY(alloc_arr(s, &s->v, D * N));
  AQS_TRY(alloc_arr(s, &s->xs, D * N));
  AQS_TRY(alloc_arr(s, &s->xb, D * N));
  AQS_TRY(alloc_arr(s, &s->fref, D * N));
  AQS_TRY(alloc_arr(s, &s->dl, D * N));
  AQS_TRY(alloc_arr(s, &s->tmp, 3 * D * N));
  AQS_TRY(alloc_arr(s, &s->d_dg, s->R));
  AQS_TRY(alloc_arr(s, &s->ubuf, D * s->nmax));
  AQS_TRY(alloc_arr(s, &s->ubuf2, D * s->nmax));
  AQS_TRY(alloc_arr(s, &s->type, N));
  AQS_TRY(alloc_arr(s, &s->perm, N));
  AQS_TRY(alloc_arr(s, &s->inv, N));
  AQS_TRY(alloc_arr(s, &s->cell, N));
  AQS_TRY(alloc_arr(s, &s->key, N));
  AQS_TRY(alloc_arr(s, &s->itmp, 3 * N));
  AQS_TRY(alloc_arr(s, &s->nnb, N));
  AQS_TRY(alloc_arr(s, &s->order, N));
  AQS_TRY(alloc_arr(s, &s->overflow, s->R));
  AQS_TRY(alloc_arr(s, &s->d_jobs, std::max(s->R, 64)));
  AQS_TRY(alloc_arr(s, &s->d_cmp, std::max(s->R, 64)));
  AQS_TRY(alloc_arr(s, &s->d_partial, 2 * (energy_blocks((int)s->nmax) + 1)));
  AQS_TRY(alloc_arr(s, &s->d_i64, 4 * std::max(s->R, 64)));
  AQS_TRY(alloc_arr(s, &s->d_shift, std::max(s->R, 64)));
  AQS_TRY(alloc_arr(s, &s->d_nnbsum, s->R));
  AQS_TRY(alloc_arr(s, &s->pubg, (size_t)N * (D == 2 ? 2 : 4)));
  CUDA_TRY(cudaEventCreate(&s->ev0));
  CUDA_TRY(cudaEventCreate(&s->ev1));
  CUDA_TRY(cudaMemsetAsync(s->v, 0, sizeof(double) * D * N, s->stream));
  CUDA_TRY(cudaMemsetAsync(s->dl, 0, sizeof(double) * D * N, s->stream));
  CUDA_TRY(cudaMemsetAsync(s->fref, 0, sizeof(double) * D * N, s->stream));
  AQS_TRY(layout_lists(s));
  return AQS_OK;
}

// Common part of system creation (positions/types uploaded by the caller).
aqs_status init_system(aqs_system* s, int dim, int R, const int64_t* n, const aqs_potential& pot,
                       int prec, double skin, int cap, int C_override, cudaStream_t stream,
                       void* (*ua)(size_t, void*), void (*uf)(void*, void*), void* actx) {
  s->dim = dim;
  s->R = R;
  s->nt = pot.n_types;
  s->pot = pot;
  s->prec = prec;
  s->skin = skin > 0.0 ? skin : 0.3;
  s->cap = cap > 0 ? cap : (dim == 2 ? 64 : 160);
  s->C_override = C_override;
  s->stream = stream;
  s->ualloc = ua;
  s->ufree = uf;
  s->actx = actx;
  s->n.assign(n, n + R);
  s->off.resize(R);
  s->ntot = 0;
  s->nmax = 0;
  for (int r = 0; r < R; r++) {
    s->off[r] = s->ntot;
    s->ntot += n[r];
    s->nmax = std::max(s->nmax, n[r]);
  }
  make_coef(s, pot);
  {
    std::array<double, 9> id{};
    for (int a = 0; a < dim; a++) id[a * dim + a] = 1.0;
    s->frame.assign(R, id);
  }
  s->geom.assign(R, RepGeom{});
  s->st.assign(R, RepState{});
  s->mean_nb.assign(R, 0.0);
  s->nnb_sum.assign(R, 0);
  for (int r = 0; r < R; r++) {
    RepGeom& g = s->geom[r];
    g.off = s->off[r];
    g.n = (int)n[r];
    int C = C_override > 0 ? C_override
                           : auto_cluster(dim, prec == AQS_MIXED, R, n[r], s->nt, s->cap);
    C = std::max(1, std::min(C, kMaxCluster));
    g.C = C;
    g.npc = (int)((n[r] + C - 1) / C);
    s->st[r].status = AQS_OK;
  }
  AQS_TRY(alloc_system(s));
  CUDA_TRY(cudaMemcpyAsync(s->d_coef, s->coef, sizeof(s->coef), cudaMemcpyHostToDevice, stream));
  std::vector<int32_t> rep_of(s->ntot), ident(s->ntot);
  for (int r = 0; r < R; r++)
    for (int64_t i = 0; i < n[r]; i++) {
      rep_of[s->off[r] + i] = r;
      ident[s->off[r] + i] = (int32_t)i;
    }
  CUDA_TRY(cudaMemcpyAsync(s->d_rep_of, rep_of.data(), sizeof(int32_t) * s->ntot,
                           cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(s->perm, ident.data(), sizeof(int32_t) * s->ntot,
                           cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(s->inv, ident.data(), sizeof(int32_t) * s->ntot,
                           cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  AQS_TRY(upload_state(s));
  return AQS_OK;
}

aqs_status check_box(aqs_system* s, int r, const double* H) {
  const int D = s->dim;
  for (int a = 0; a < D; a++)
    for (int b = 0; b < a; b++)
      if (H[a * D + b] != 0.0) return fail(AQS_ERR_INVALID_ARG, "cell must be upper triangular");
  if (D == 3 && (H[0 * 3 + 2] != 0.0 || H[1 * 3 + 2] != 0.0))
    return fail(AQS_ERR_UNSUPPORTED, "3D cells may only tilt in xy");
  for (int a = 0; a < D; a++)
    if (!(H[a * D + a] > 0.0)) return fail(AQS_ERR_INVALID_ARG, "cell diagonal must be positive");
  double w[3];
  cell_widths(D, H, w);
  for (int c = 0; c < D; c++)
    if (!(s->rlist * 3.0 <= w[c]))
      return fail(AQS_ERR_BOX_TOO_SMALL, "replica %d: width %.4g < 3 (rc+skin) = %.4g", r, w[c],
                  3.0 * s->rlist);
  return AQS_OK;
}

// Copy user-order positions (host or device) of replica r into the system.
// Non-finite coordinates are refused (AQS_ERR_NONFINITE) before anything is
// written; device inputs are checked on a host copy.
aqs_status put_positions(aqs_system* s, int r, const double* pos) {
  const int D = s->dim;
  const size_t cnt = (size_t)D * s->n[r];
  size_t bytes = sizeof(double) * cnt;
  const double* src = pos;
  const bool dev = is_device_ptr(pos);
  std::vector<double> hcopy;
  const double* hp = pos;
  if (dev) {
    hcopy.resize(cnt);
    CUDA_TRY(cudaMemcpyAsync(hcopy.data(), pos, bytes, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    hp = hcopy.data();
  }
  for (size_t k = 0; k < cnt; k++)
    if (!std::isfinite(hp[k]))
      return fail(AQS_ERR_NONFINITE, "replica %d: position component %zu is not finite", r, k);
  if (!dev) {
    CUDA_TRY(cudaMemcpyAsync(s->ubuf, pos, bytes, cudaMemcpyHostToDevice, s->stream));
    src = s->ubuf;
  }
  CUDA_TRY(launch_scatter_user(src, s->x, s->ntot, s->off[r], (int)s->n[r], s->perm, D, s->stream));
  CUDA_TRY(cudaMemsetAsync(s->v, 0, sizeof(double) * D * s->ntot, s->stream));
  return AQS_OK;
}

aqs_status fetch_positions(const aqs_system* s, int r, double* out) {
  const int D = s->dim;
  bool dev = is_device_ptr(out);
  double* dst = dev ? out : s->ubuf;
  CUDA_TRY(launch_gather_user(s->x, s->ntot, s->off[r], (int)s->n[r], s->perm, D, dst, s->stream));
  if (!dev)
    CUDA_TRY(cudaMemcpyAsync(out, s->ubuf, sizeof(double) * D * s->n[r], cudaMemcpyDeviceToHost,
                             s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return AQS_OK;
}

void destroy(aqs_system* s) {
  if (!s) return;
  if (s->chains) destroy(s->chains);
  cudaStreamSynchronize(s->stream);
  if (s->ev0) cudaEventDestroy(s->ev0);
  if (s->ev1) cudaEventDestroy(s->ev1);
  for (int k = 0; k < 4; k++)
    if (s->aux[k]) {
      cudaStreamSynchronize(s->aux[k]);
      cudaStreamDestroy(s->aux[k]);
    }
  for (int k = 0; k < 5; k++)
    if (s->aux_ev[k]) cudaEventDestroy(s->aux_ev[k]);
  for (auto& a : s->allocs) {
    if (s->ufree) s->ufree(a.p, s->actx);
    else cudaFree(a.p);
  }
  s->allocs.clear();
  delete s;
}

// ---- two-level parallel stepping (Algorithm 1) ----
aqs_status ensure_chains(aqs_system* s, int src, int P) {
  if (s->chains && s->chains->R == P && s->chains->n[0] == s->n[src]) return AQS_OK;
  if (s->chains) destroy(s->chains);
  s->chains = nullptr;
  aqs_system* c = new aqs_system();
  std::vector<int64_t> n(P, s->n[src]);
  aqs_status st = init_system(c, s->dim, P, n.data(), s->pot, s->prec, s->skin, s->cap, 0,
                              s->stream, s->ualloc, s->ufree, s->actx);
  if (st != AQS_OK) {
    destroy(c);
    return st;
  }
  const size_t per = (size_t)s->dim * s->n[src];
  c->snap = static_cast<double*>(dalloc(c, sizeof(double) * per * P));
  c->ends = static_cast<double*>(dalloc(c, sizeof(double) * per * P));
  if (!c->snap || !c->ends) {
    destroy(c);
    return fail(AQS_ERR_OOM, "chain snapshot allocation failed");
  }
  c->tune_iters = s->tune_iters;
  c->launch_budget = s->launch_budget;
  c->staging = s->staging_user ? s->staging : -1;
  c->staging_user = s->staging_user;
  c->tpa = s->tpa_user ? s->tpa : 1;
  c->tpa_user = s->tpa_user;
  c->grid_barrier = s->grid_barrier_user ? s->grid_barrier : false;
  c->grid_barrier_user = s->grid_barrier_user;
  s->chains = c;
  return AQS_OK;
}

// Copies replica `sr` of system a into replicas `drs` of system b, the copy k
// sheared by shift[k], or (maps non-null: host [ncopy][9]) mapped by the
// upper-triangular maps[k] into the cell cells[k] (host [ncopy][9], 3 x 3
// slots); velocities cleared.  Lists are not copied (rebuilt).
aqs_status copy_replicas(aqs_system* a, int sr, aqs_system* b, const std::vector<int>& drs,
                         const std::vector<double>& shift, const double* maps = nullptr,
                         const double* cells = nullptr) {
  RepCopy c;
  c.sx = a->x;
  c.sxb = a->xb;
  c.stype = a->type;
  c.sperm = a->perm;
  c.sinv = a->inv;
  c.scell = a->cell;
  c.snnb = a->nnb;
  c.snb = a->nb;
  c.sN = a->ntot;
  c.soff = a->off[sr];
  c.snb_off = a->geom[sr].nb_off;
  c.dx = b->x;
  c.dxb = b->xb;
  c.dv = b->v;
  c.dtype = b->type;
  c.dperm = b->perm;
  c.dinv = b->inv;
  c.dcell = b->cell;
  c.dnnb = b->nnb;
  c.dnb = b->nb;
  c.dN = b->ntot;
  std::vector<int64_t> offs(2 * drs.size());
  for (size_t k = 0; k < drs.size(); k++) {
    offs[k] = b->off[drs[k]];
    offs[drs.size() + k] = b->geom[drs[k]].nb_off;
  }
  CUDA_TRY(cudaMemcpyAsync(b->d_i64, offs.data(), sizeof(int64_t) * offs.size(),
                           cudaMemcpyHostToDevice, b->stream));
  CUDA_TRY(cudaMemcpyAsync(b->d_shift, shift.data(), sizeof(double) * shift.size(),
                           cudaMemcpyHostToDevice, b->stream));
  c.doff = b->d_i64;
  c.dnb_off = b->d_i64 + drs.size();
  c.shift = b->d_shift;
  c.maps = nullptr;
  if (maps) {
    if (!b->d_maps) AQS_TRY(alloc_arr(b, &b->d_maps, (size_t)9 * b->R));
    CUDA_TRY(cudaMemcpyAsync(b->d_maps, maps, sizeof(double) * 9 * drs.size(),
                             cudaMemcpyHostToDevice, b->stream));
    c.maps = b->d_maps;
  }
  c.n = (int)a->n[sr];
  c.cap = 0;  // lists are rebuilt for the new owner layout
  c.ncopy = (int)drs.size();
  c.D = a->dim;
  CUDA_TRY(launch_copy_rep(c, b->stream));
  const int D = a->dim;
  for (size_t k = 0; k < drs.size(); k++) {
    RepGeom& g = b->geom[drs[k]];
    std::memcpy(g.H, a->geom[sr].H, sizeof(g.H));
    if (cells) {
      for (int x = 0; x < D; x++)
        for (int y = 0; y < D; y++) g.H[x * D + y] = cells[9 * k + x * 3 + y];
    } else {
      g.H[0 * D + 1] += shift[k] * g.H[1 * D + 1];
    }
  }
  std::vector<uint8_t> flags(b->R, 0);
  for (int r : drs) flags[r] = 1;
  return rebuild(b, flags);
}

// ---- deformation histories (pure / pull-push shear, cyclic protocols) ----
// The stored cell H is always upper triangular; the laboratory cell is Q H
// with Q the replica's frame.  An increment F acts on the laboratory cell
// (Eq. 1 with a general matrix): H_lab <- F H_lab, Q <- Gram-Schmidt frame of
// the new H_lab, H <- Q^T H_lab, and stored positions move by the
// upper-triangular M = Q_new^T F Q_old (Eq. 3 in the two frames).  For
// simple shear Q stays the identity and M = F.

// Columns q_c of the Gram-Schmidt frame of G (d x d, row-major): G = Q R,
// R upper triangular with a positive diagonal.  Q is row-major d x d.
void gs_frame(int D, const double* G, double* Q) {
  double q[3][3] = {{0.0}};
  double n0 = 0.0;
  for (int a = 0; a < D; a++) n0 += G[a * D] * G[a * D];
  n0 = std::sqrt(n0);
  for (int a = 0; a < D; a++) q[0][a] = G[a * D] / n0;
  double p = 0.0;
  for (int a = 0; a < D; a++) p += q[0][a] * G[a * D + 1];
  double n1 = 0.0;
  for (int a = 0; a < D; a++) {
    q[1][a] = G[a * D + 1] - p * q[0][a];
    n1 += q[1][a] * q[1][a];
  }
  n1 = std::sqrt(n1);
  for (int a = 0; a < D; a++) q[1][a] /= n1;
  if (D == 3) {
    q[2][0] = q[0][1] * q[1][2] - q[0][2] * q[1][1];
    q[2][1] = q[0][2] * q[1][0] - q[0][0] * q[1][2];
    q[2][2] = q[0][0] * q[1][1] - q[0][1] * q[1][0];
  }
  for (int a = 0; a < D; a++)
    for (int c = 0; c < D; c++) Q[a * D + c] = q[c][a];
}

// One increment F from the frame Q and stored cell H (both updated); writes
// the map M and the new cell in 3 x 3 slots.
void hist_step(int D, double* Q, double* H, const double* F, double* M9, double* H9) {
  double L[9], Ln[9], Qn[9], T[9];
  for (int a = 0; a < D; a++)
    for (int c = 0; c < D; c++) {
      double v = 0.0;
      for (int k = 0; k < D; k++) v += Q[a * D + k] * H[k * D + c];
      L[a * D + c] = v;
    }
  for (int a = 0; a < D; a++)
    for (int c = 0; c < D; c++) {
      double v = 0.0;
      for (int k = 0; k < D; k++) v += F[a * D + k] * L[k * D + c];
      Ln[a * D + c] = v;
    }
  gs_frame(D, Ln, Qn);
  for (int a = 0; a < D; a++)  // T = F Q_old
    for (int c = 0; c < D; c++) {
      double v = 0.0;
      for (int k = 0; k < D; k++) v += F[a * D + k] * Q[k * D + c];
      T[a * D + c] = v;
    }
  for (int k = 0; k < 9; k++) M9[k] = H9[k] = 0.0;
  for (int a = 0; a < D; a++)
    for (int c = a; c < D; c++) {
      double m = 0.0, h = 0.0;
      for (int k = 0; k < D; k++) {
        m += Qn[k * D + a] * T[k * D + c];
        h += Qn[k * D + a] * Ln[k * D + c];
      }
      M9[a * 3 + c] = m;
      H9[a * 3 + c] = h;
    }
  for (int a = 0; a < D; a++)
    for (int c = 0; c < D; c++) H[a * D + c] = H9[a * 3 + c];
  std::memcpy(Q, Qn, sizeof(double) * D * D);
}

// A cell a history reaches must keep the minimum-image rule and (3D) its
// tilt in xy only.
aqs_status check_hist_cell(aqs_system* s, const double* H) {
  const int D = s->dim;
  if (D == 3 && (std::fabs(H[2]) > 0.0 || std::fabs(H[5]) > 0.0))
    return fail(AQS_ERR_UNSUPPORTED, "3D deformation histories must keep the cell tilted in xy only");
  if (!(H[0] > 0.0) || !(H[D + 1] > 0.0) || (D == 3 && !(H[8] > 0.0)))
    return fail(AQS_ERR_INVALID_ARG, "deformation history inverts the cell");
  double w[3];
  cell_widths(D, H, w);
  for (int c = 0; c < D; c++)
    if (!(s->rlist * 3.0 <= w[c]))
      return fail(AQS_ERR_BOX_TOO_SMALL, "deformation history: width %.4g < 3 (rc+skin) = %.4g",
                  w[c], 3.0 * s->rlist);
  return AQS_OK;
}

// Job table of one replica for n increments F[0..n) (d x d each) from (Q, H),
// both advanced; with first_noaffine the job's step 0 has no increment (row
// left as the identity map into the current cell).  Optionally returns the
// product of the maps (3 x 3 slots).
aqs_status hist_table(aqs_system* s, double* Q, double* H, const double* F, int64_t n,
                      bool first_noaffine, std::vector<double>& table, double* Mprod = nullptr) {
  const int D = s->dim;
  const int64_t rows = n + (first_noaffine ? 1 : 0);
  table.assign((size_t)rows * kHistFields, 0.0);
  double P[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  int64_t row = 0;
  if (first_noaffine) {
    for (int a = 0; a < 3; a++) table[a * 3 + a] = 1.0;
    for (int a = 0; a < D; a++)
      for (int c = 0; c < D; c++) table[9 + a * 3 + c] = H[a * D + c];
    row = 1;
  }
  for (int64_t k = 0; k < n; k++, row++) {
    double* r = table.data() + row * kHistFields;
    hist_step(D, Q, H, F + (size_t)k * D * D, r, r + 9);
    if (D == 2) r[8] = 1.0;  // unused z slot of the map: identity
    AQS_TRY(check_hist_cell(s, H));
    double Pn[9] = {0};
    for (int a = 0; a < 3; a++)
      for (int c = 0; c < 3; c++)
        for (int k2 = 0; k2 < 3; k2++) Pn[a * 3 + c] += r[a * 3 + k2] * P[k2 * 3 + c];
    std::memcpy(P, Pn, sizeof(P));
  }
  if (Mprod) std::memcpy(Mprod, P, sizeof(P));
  return AQS_OK;
}

aqs_status gather_user(aqs_system* s, int r, double* dst) {
  CUDA_TRY(launch_gather_user(s->x, s->ntot, s->off[r], (int)s->n[r], s->perm, s->dim, dst,
                              s->stream));
  return AQS_OK;
}

}  // namespace

// =====================================================================
//                                C ABI
// =====================================================================
extern "C" {

void aqs_fire_params_default(aqs_fire_params* f) {
  if (!f) return;
  f->dt0 = 0.005;
  f->alpha0 = 0.1;
  f->f_inc = 1.1;
  f->f_dec = 0.5;
  f->f_alpha = 0.99;
  f->dt_max = 0.05;
  f->dt_min = 1e-4;
  f->max_step = 0.1;
  f->tol = 1e-10;
  f->n_min = 5;
  f->max_iter = 1000000;
  f->ref_ratio = 30.0;
  f->ref_dmax = 0.05;
}

aqs_status aqs_create_system(const aqs_system_desc* d, aqs_system** out) {
  if (!d || !out) return fail(AQS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return fail(AQS_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (d->n_replicas < 1 || !d->n_atoms || !d->box || !d->pos || !d->types)
    return fail(AQS_ERR_INVALID_ARG, "missing replica data");
  if (d->pot.n_types < 1 || d->pot.n_types > AQS_MAX_TYPES || !(d->pot.rc_factor > 0.0))
    return fail(AQS_ERR_INVALID_ARG, "bad potential");
  for (int k = 0; k < d->pot.n_types * d->pot.n_types; k++)
    if (!(d->pot.sigma[k] > 0.0) || !(d->pot.eps[k] >= 0.0))
      return fail(AQS_ERR_INVALID_ARG, "sigma must be > 0 and eps >= 0");
  if (d->precision != AQS_FP64 && d->precision != AQS_MIXED)
    return fail(AQS_ERR_INVALID_ARG, "bad precision");
  int64_t ntot = 0;
  for (int r = 0; r < d->n_replicas; r++) {
    if (d->n_atoms[r] < 2 || d->n_atoms[r] > 16 * 4096)
      return fail(AQS_ERR_UNSUPPORTED, "replica %d: atom count %lld outside [2, 65536]", r,
                  (long long)d->n_atoms[r]);
    ntot += d->n_atoms[r];
  }
  if (d->cluster_size > kMaxCluster) return fail(AQS_ERR_INVALID_ARG, "cluster_size > 16");
  aqs_system* s = new aqs_system();
  aqs_status st = init_system(s, d->dim, d->n_replicas, d->n_atoms, d->pot, d->precision, d->skin,
                              d->nlist_capacity, d->cluster_size, (cudaStream_t)d->stream,
                              d->alloc, d->free, d->alloc_ctx);
  if (st != AQS_OK) {
    destroy(s);
    return st;
  }
  for (int r = 0; r < s->R; r++) {
    const int64_t npc = s->geom[r].npc;
    if (npc > 4096) {
      destroy(s);
      return fail(AQS_ERR_UNSUPPORTED, "replica %d: %lld atoms per CTA exceeds 4096", r,
                  (long long)npc);
    }
    std::memcpy(s->geom[r].H, d->box + (size_t)r * d->dim * d->dim,
                sizeof(double) * d->dim * d->dim);
    st = check_box(s, r, s->geom[r].H);
    if (st != AQS_OK) {
      destroy(s);
      return st;
    }
    s->geom[r].tilt_b = s->geom[r].H[1];
  }
  // types (validated on the host)
  std::vector<int32_t> ht(ntot);
  if (is_device_ptr(d->types)) {
    if (cudaMemcpy(ht.data(), d->types, sizeof(int32_t) * ntot, cudaMemcpyDeviceToHost) != cudaSuccess) {
      destroy(s);
      return fail(AQS_ERR_CUDA, "reading types failed");
    }
  } else {
    std::memcpy(ht.data(), d->types, sizeof(int32_t) * ntot);
  }
  for (int64_t i = 0; i < ntot; i++)
    if (ht[i] < 0 || ht[i] >= s->nt) {
      destroy(s);
      return fail(AQS_ERR_INVALID_ARG, "type %d of atom %lld out of range", ht[i], (long long)i);
    }
  if (cudaMemcpyAsync(s->type, ht.data(), sizeof(int32_t) * ntot, cudaMemcpyHostToDevice,
                      s->stream) != cudaSuccess) {
    destroy(s);
    return fail(AQS_ERR_CUDA, "uploading types failed");
  }
  bool dev = is_device_ptr(d->pos);
  for (int r = 0; r < s->R; r++) {
    const double* p = d->pos + (size_t)s->off[r] * s->dim;
    (void)dev;
    st = put_positions(s, r, p);
    if (st != AQS_OK) {
      destroy(s);
      return st;
    }
  }
  st = rebuild_all(s);
  if (st != AQS_OK) {
    destroy(s);
    return st;
  }
  *out = s;
  return AQS_OK;
}

void aqs_destroy_system(aqs_system* s) { destroy(s); }

aqs_status aqs_affine_shear(aqs_system* s, const double* dgamma) {
  if (!s || !dgamma) return fail(AQS_ERR_INVALID_ARG, "null argument");
  std::vector<double> dg(dgamma, dgamma + s->R);
  for (int r = 0; r < s->R; r++) {
    if (!std::isfinite(dg[r])) return fail(AQS_ERR_INVALID_ARG, "non-finite dgamma");
    double H[9];
    std::memcpy(H, s->geom[r].H, sizeof(H));
    H[1] += dg[r] * H[s->dim + 1];
    double w[3];
    cell_widths(s->dim, H, w);
    if (!(s->rlist * 3.0 <= w[0])) return fail(AQS_ERR_BOX_TOO_SMALL, "tilt too large");
  }
  return affine_impl(s, dg);
}

aqs_status aqs_minimize(aqs_system* s, const aqs_fire_params* f, const uint8_t* mask,
                        aqs_min_result* out) {
  if (!s || !f) return fail(AQS_ERR_INVALID_ARG, "null argument");
  if (!(f->tol > 0.0) || !(f->dt0 > 0.0) || f->max_iter < 0 || !(f->max_step > 0.0))
    return fail(AQS_ERR_INVALID_ARG, "bad FIRE parameters");
  std::vector<uint8_t> m(s->R, 1);
  if (mask)
    for (int r = 0; r < s->R; r++) m[r] = mask[r] != 0;
  return minimize_impl(s, f, m, out);
}

aqs_status aqs_run_sequential(aqs_system* s, const aqs_fire_params* f, double dgamma,
                              int64_t n_steps, double* energy, double* tau, int64_t* fire_iters,
                              double* nonaffine_out) {
  if (!s || !f || n_steps < 0 || !std::isfinite(dgamma))
    return fail(AQS_ERR_INVALID_ARG, "bad argument");
  if (n_steps == 0) return AQS_OK;
  for (int r = 0; r < s->R; r++) {
    double H[9];
    std::memcpy(H, s->geom[r].H, sizeof(H));
    H[1] += n_steps * dgamma * H[s->dim + 1];
    double w[3];
    cell_widths(s->dim, H, w);
    if (!(s->rlist * 3.0 <= w[0])) return fail(AQS_ERR_BOX_TOO_SMALL, "tilt too large");
  }
  std::vector<Job> jobs(s->R);
  for (int r = 0; r < s->R; r++) {
    jobs[r].nsteps = n_steps;
    jobs[r].dgamma = dgamma;
  }
  JobOut out;
  AQS_TRY(run_jobs(s, f, jobs, &out));
  for (int64_t k = 0; k < n_steps; k++)
    for (int r = 0; r < s->R; r++) {
      const double* rec = &out.rec[((size_t)r * out.stride + k) * kRecFields];
      size_t i = (size_t)k * s->R + r;
      if (energy) energy[i] = rec[0];
      if (tau) tau[i] = rec[1];
      if (fire_iters) fire_iters[i] = (int64_t)rec[3];
      if (nonaffine_out) nonaffine_out[i] = rec[2];
    }
  return AQS_OK;
}

aqs_status aqs_deform(aqs_system* s, const double* F) {
  if (!s || !F) return fail(AQS_ERR_INVALID_ARG, "null argument");
  const int D = s->dim;
  std::vector<double> maps((size_t)9 * s->R), cells((size_t)9 * s->R);
  std::vector<std::array<double, 9>> fr(s->frame);
  std::vector<uint8_t> flags(s->R, 1);
  for (int r = 0; r < s->R; r++) {
    for (int k = 0; k < D * D; k++)
      if (!std::isfinite(F[(size_t)r * D * D + k])) return fail(AQS_ERR_INVALID_ARG, "non-finite F");
    double H[9];
    std::memcpy(H, s->geom[r].H, sizeof(H));
    hist_step(D, fr[r].data(), H, F + (size_t)r * D * D, &maps[9 * r], &cells[9 * r]);
    if (D == 2) maps[9 * r + 8] = 1.0;
    AQS_TRY(check_hist_cell(s, H));  // nothing applied yet
  }
  if (!s->d_maps) AQS_TRY(alloc_arr(s, &s->d_maps, (size_t)9 * s->R));
  CUDA_TRY(cudaMemcpyAsync(s->d_maps, maps.data(), sizeof(double) * maps.size(),
                           cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(cudaMemcpyAsync(s->d_flag, flags.data(), s->R, cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(launch_deform(D, s->x, s->xb, s->d_rep_of, s->d_flag, s->d_maps, s->ntot, s->stream));
  for (int r = 0; r < s->R; r++) {
    for (int a = 0; a < D; a++)
      for (int c = 0; c < D; c++) s->geom[r].H[a * D + c] = cells[9 * r + a * 3 + c];
    s->frame[r] = fr[r];
  }
  sync_tilt_to_state(s);
  // the lists are rebuilt in the new cell (a stretch changes pair distances
  // without changing the tilt the simple-shear skin test watches)
  return rebuild(s, flags);
}

aqs_status aqs_run_history(aqs_system* s, const aqs_fire_params* f, const double* F,
                           int64_t n_steps, double* energy, double* tau, int64_t* fire_iters,
                           double* nonaffine_out) {
  if (!s || !f || n_steps < 0 || (n_steps > 0 && !F)) return fail(AQS_ERR_INVALID_ARG, "bad argument");
  if (n_steps == 0) return AQS_OK;
  const int D = s->dim;
  for (int64_t k = 0; k < n_steps * D * D; k++)
    if (!std::isfinite(F[k])) return fail(AQS_ERR_INVALID_ARG, "non-finite F");
  std::vector<Job> jobs(s->R);
  std::vector<std::array<double, 9>> fr(s->frame);
  for (int r = 0; r < s->R; r++) {
    double H[9];
    std::memcpy(H, s->geom[r].H, sizeof(H));
    AQS_TRY(hist_table(s, fr[r].data(), H, F, n_steps, false, jobs[r].table));
    jobs[r].nsteps = n_steps;
  }
  JobOut out;
  AQS_TRY(run_jobs(s, f, jobs, &out));
  for (int r = 0; r < s->R; r++) s->frame[r] = fr[r];
  AQS_TRY(rebuild_all(s));  // lists at the final cell for later simple-shear calls
  for (int64_t k = 0; k < n_steps; k++)
    for (int r = 0; r < s->R; r++) {
      const double* rec = &out.rec[((size_t)r * out.stride + k) * kRecFields];
      size_t i = (size_t)k * s->R + r;
      if (energy) energy[i] = rec[0];
      if (tau) tau[i] = rec[1];
      if (fire_iters) fire_iters[i] = (int64_t)rec[3];
      if (nonaffine_out) nonaffine_out[i] = rec[2];
    }
  return AQS_OK;
}

aqs_status aqs_get_frame(const aqs_system* s, int r, double* Q) {
  if (!s || !Q || r < 0 || r >= s->R) return fail(AQS_ERR_INVALID_ARG, "bad argument");
  std::memcpy(Q, s->frame[r].data(), sizeof(double) * s->dim * s->dim);
  return AQS_OK;
}

aqs_status aqs_parallel_step(aqs_system* s, int src, const aqs_fire_params* f,
                             const aqs_parallel_params* p, aqs_parallel_result* out) {
  if (!s || !f || !p || !out) return fail(AQS_ERR_INVALID_ARG, "null argument");
  if (src < 0 || src >= s->R) return fail(AQS_ERR_INVALID_ARG, "replica out of range");
  if (p->K < 1 || p->P < 1 || p->n_steps < 0 || !std::isfinite(p->dgamma))
    return fail(AQS_ERR_INVALID_ARG, "bad parallel parameters");
  if (p->warm_start) return fail(AQS_ERR_UNSUPPORTED, "warm start is not available");
  const double* Fh = p->F_steps;  // deformation history of this call (nullable)
  if (Fh)
    for (int64_t k = 0; k < p->n_steps * s->dim * s->dim; k++)
      if (!std::isfinite(Fh[k])) return fail(AQS_ERR_INVALID_ARG, "non-finite F_steps");
  const double eq_tol = p->eq_tol > 0.0 ? p->eq_tol : 1e-6;
  const double ev_thr = p->event_threshold > 0.0 ? p->event_threshold : 1e-2;
  const int P = p->P, D = s->dim;
  // dynamic K (K_max > K): the chain length of the next pass is doubled after
  // a pass without a failed test, up to K_max, and ceil(q / P) after a failed
  // test, q the steps the pass accepted (the same rule as the oracle's)
  const bool adaptive = p->K_max > p->K;
  const int Kcap = adaptive ? p->K_max : p->K;
  int K = p->K;
  const int n = (int)s->n[src];
  AQS_TRY(ensure_chains(s, src, P));
  aqs_system* c = s->chains;
  out->iterations = out->accepted_steps = out->rejections = 0;
  out->fire_iters_total = out->evals64_total = 0;
  out->chains_stopped = 0;
  out->K_next = p->K;
  out->n_log = 0;
  std::vector<double> cE((size_t)P * Kcap), cT((size_t)P * Kcap), cD((size_t)P * Kcap);
  std::vector<int64_t> cI((size_t)P * Kcap);
  int64_t n_cur = 0;
  const size_t per = (size_t)D * n;
  while (n_cur < p->n_steps && (p->max_iterations <= 0 || out->iterations < p->max_iterations)) {
    const int64_t rem = p->n_steps - n_cur;
    if (out->K_pass && out->iterations < p->n_steps) out->K_pass[out->iterations] = K;
    const int P_eff = (int)std::min<int64_t>(P, (rem + K - 1) / K);
    std::vector<int> Ki(P_eff, K);
    if (rem < (int64_t)P_eff * K) Ki[P_eff - 1] = (int)(rem - (int64_t)(P_eff - 1) * K);
    // level I: r^c_iK = F^(i K dgamma) r_star (Eq. 18)
    std::vector<int> drs(P_eff);
    std::vector<double> shift(P_eff);
    for (int i = 0; i < P_eff; i++) {
      drs[i] = i;
      shift[i] = (double)i * K * p->dgamma;
    }
    std::vector<Job> jobs(P);
    std::vector<std::array<double, 9>> chain_frame(P_eff);
    if (Fh) {
      // level I under a history: chain i starts after the i K increments
      // that follow the current step, applied one after the other (the
      // sequence chain i-1 applies on its way), so that chain i starts in
      // exactly the cell where chain i-1 ends; its job table continues the
      // sequence with its own K_i increments
      const int DD = D * D;
      std::vector<double> maps((size_t)9 * P_eff), cells((size_t)9 * P_eff);
      for (int i = 0; i < P_eff; i++) {
        std::array<double, 9> Q = s->frame[src];
        double H[9];
        std::memcpy(H, s->geom[src].H, sizeof(H));
        std::vector<double> lvl1;
        AQS_TRY(hist_table(s, Q.data(), H, Fh + (size_t)n_cur * DD, (int64_t)i * K, false, lvl1,
                           &maps[9 * i]));
        for (int k = 0; k < 9; k++) cells[9 * i + k] = 0.0;
        for (int a = 0; a < D; a++)
          for (int cc = 0; cc < D; cc++) cells[9 * i + a * 3 + cc] = H[a * D + cc];
        c->frame[i] = Q;
        AQS_TRY(hist_table(s, Q.data(), H, Fh + (size_t)(n_cur + (int64_t)i * K) * DD, Ki[i],
                           true, jobs[i].table));
        chain_frame[i] = Q;
      }
      AQS_TRY(copy_replicas(s, src, c, drs, shift, maps.data(), cells.data()));
    } else {
      AQS_TRY(copy_replicas(s, src, c, drs, shift));
    }
    // level II (Eq. 19): chain i runs F once (its outgoing configuration,
    // kept as a caller-order snapshot for i >= 1) and then K_i fine AQS
    // steps, all inside persistent launches; chains never wait for each other
    // between fine steps
    for (int i = 0; i < P_eff; i++) {
      jobs[i].nsteps = 1 + Ki[i];
      jobs[i].dgamma = p->dgamma;
      jobs[i].first_noaffine = 1;
      jobs[i].want_snap = i >= 1;
    }
    // Equality tests (Eq. 20): end of chain i-1 vs F(r^c_iK), the snapshot
    // of chain i after its first minimisation.  A test is made as soon as
    // both are available (between persistent-launch passes); once a test i
    // fails, chains i.. are discarded whatever the earlier tests give, so
    // unless run_discarded is set they stop there and their SMs go to the
    // chains that are still needed.  Decisions are the same either way.
    std::vector<double> m(P_eff, 0.0);
    std::vector<uint8_t> known(P_eff, 0), dropped;
    auto run_tests = [&](const std::vector<uint8_t>& running) -> aqs_status {
      std::vector<CmpJob> cj;
      std::vector<int> idx;
      for (int i = 1; i < P_eff; i++) {
        if (known[i] || running[i - 1] || c->st[i - 1].status != AQS_OK || c->st[i].step < 1)
          continue;
        AQS_TRY(gather_user(c, i - 1, c->ends + per * (i - 1)));
        CmpJob J;
        J.a = c->ends + per * (i - 1);
        J.b = c->d_snap + (size_t)c->dim * c->nmax * i;
        J.sa = D;
        J.sc = 1;
        J.sb = D;
        J.sc2 = 1;
        std::memcpy(J.H, c->geom[i - 1].H, sizeof(J.H));  // both at strain i K dgamma
        J.n = n;
        cj.push_back(J);
        idx.push_back(i);
      }
      if (cj.empty()) return AQS_OK;
      std::vector<double> v(cj.size());
      CUDA_TRY(cudaMemcpyAsync(c->d_jobs, cj.data(), sizeof(CmpJob) * cj.size(),
                               cudaMemcpyHostToDevice, c->stream));
      CUDA_TRY(launch_compare(D, c->d_jobs, (int)cj.size(), c->d_cmp, c->stream));
      CUDA_TRY(cudaMemcpyAsync(v.data(), c->d_cmp, sizeof(double) * cj.size(),
                               cudaMemcpyDeviceToHost, c->stream));
      CUDA_TRY(cudaStreamSynchronize(c->stream));
      for (size_t k = 0; k < idx.size(); k++) {
        m[idx[k]] = v[k];
        known[idx[k]] = 1;
      }
      return AQS_OK;
    };
    PassHook hook = [&](std::vector<int>& next, std::vector<uint8_t>& drop) -> aqs_status {
      std::vector<uint8_t> running(c->R, 0);
      for (int r : next) running[r] = 1;
      AQS_TRY(run_tests(running));
      int fail_at = P_eff;
      for (int i = 1; i < P_eff; i++)
        if (known[i] && !(m[i] < eq_tol)) {
          fail_at = i;
          break;
        }
      if (fail_at < P_eff) {
        std::vector<int> keep;
        for (int r : next) {
          if (r >= fail_at) drop[r] = 1;
          else keep.push_back(r);
        }
        next.swap(keep);
      }
      return AQS_OK;
    };
    JobOut jo;
    AQS_TRY(run_jobs(c, f, jobs, &jo, nullptr, p->run_discarded ? nullptr : &hook, &dropped));
    for (int i = 0; i < P_eff; i++) {
      const double* rec = &jo.rec[(size_t)i * jo.stride * kRecFields];
      // steps this chain completed (all of them unless it was stopped)
      const int64_t done = dropped[i] ? c->st[i].step : 1 + Ki[i];
      if (dropped[i]) out->chains_stopped++;
      if (done >= 1) {
        out->fire_iters_total += (int64_t)rec[3];
        out->evals64_total += (int64_t)rec[4];
      }
      for (int k = 0; k < Ki[i] && k + 1 < done; k++) {
        const double* q = rec + (size_t)(k + 1) * kRecFields;
        cE[(size_t)i * Kcap + k] = q[0];
        cT[(size_t)i * Kcap + k] = q[1];
        cD[(size_t)i * Kcap + k] = q[2];
        cI[(size_t)i * Kcap + k] = (int64_t)q[3];
        out->fire_iters_total += (int64_t)q[3];
        out->evals64_total += (int64_t)q[4];
      }
    }
    if (P_eff > 1) AQS_TRY(run_tests(std::vector<uint8_t>(c->R, 0)));
    int first_fail = -1;
    int64_t q = Ki[0];
    for (int i = 1; i < P_eff; i++) {
      if (!known[i]) return fail(AQS_ERR_CUDA, "internal: equality test %d was not made", i);
      bool eq = m[i] < eq_tol;
      if (out->n_log < out->log_cap) {
        int64_t j = out->n_log;
        if (out->log_iter) out->log_iter[j] = out->iterations;
        if (out->log_i) out->log_i[j] = i;
        if (out->log_eq) out->log_eq[j] = eq ? 1 : 0;
        if (out->log_m) out->log_m[j] = m[i];
      }
      out->n_log++;
      if (!eq) {
        first_fail = i;
        break;
      }
      q += Ki[i];
    }
    const int last = first_fail < 0 ? P_eff - 1 : first_fail - 1;
    int64_t kk = n_cur;
    for (int i = 0; i <= last; i++)
      for (int j = 0; j < Ki[i]; j++, kk++) {
        size_t src_i = (size_t)i * Kcap + j;
        if (out->energy) out->energy[kk] = cE[src_i];
        if (out->tau) out->tau[kk] = cT[src_i];
        if (out->fire_iters) out->fire_iters[kk] = cI[src_i];
        if (out->nonaffine) out->nonaffine[kk] = cD[src_i];
        if (out->event) out->event[kk] = cD[src_i] > ev_thr ? 1 : 0;
      }
    // r_star <- r_q: the end of chain `last`
    AQS_TRY(copy_replicas(c, last, s, std::vector<int>{src}, std::vector<double>{0.0}));
    if (Fh) s->frame[src] = chain_frame[last];
    n_cur += q;
    out->accepted_steps += q;
    out->iterations++;
    if (first_fail >= 0) out->rejections++;
    if (adaptive)
      K = first_fail < 0 ? std::min(Kcap, 2 * K)
                         : (int)std::max<int64_t>(1, (q + P - 1) / P);
  }
  out->K_next = K;
  return AQS_OK;
}

aqs_status aqs_compare_configs(const aqs_system* a, int ra, const aqs_system* b, int rb,
                               double tol, double* max_disp, int* equal) {
  if (!a || !b) return fail(AQS_ERR_INVALID_ARG, "null system");
  if (ra < 0 || ra >= a->R || rb < 0 || rb >= b->R) return fail(AQS_ERR_INVALID_ARG, "bad replica");
  if (a->n[ra] != b->n[rb] || a->dim != b->dim)
    return fail(AQS_ERR_INVALID_ARG, "replicas differ in size or dimension");
  aqs_system* sa = const_cast<aqs_system*>(a);
  aqs_system* sb = const_cast<aqs_system*>(b);
  CUDA_TRY(cudaStreamSynchronize(sb->stream));
  AQS_TRY(gather_user(sa, ra, sa->ubuf));
  AQS_TRY(gather_user(sb, rb, sa->ubuf2));
  CUDA_TRY(cudaStreamSynchronize(sb->stream));
  CmpJob J;
  J.a = sa->ubuf;
  J.b = sa->ubuf2;
  J.sa = a->dim;
  J.sc = 1;
  J.sb = a->dim;
  J.sc2 = 1;
  std::memcpy(J.H, a->geom[ra].H, sizeof(J.H));
  J.n = (int)a->n[ra];
  CUDA_TRY(cudaMemcpyAsync(sa->d_jobs, &J, sizeof(J), cudaMemcpyHostToDevice, sa->stream));
  CUDA_TRY(launch_compare(a->dim, sa->d_jobs, 1, sa->d_cmp, sa->stream));
  double m = 0.0;
  CUDA_TRY(cudaMemcpyAsync(&m, sa->d_cmp, sizeof(double), cudaMemcpyDeviceToHost, sa->stream));
  CUDA_TRY(cudaStreamSynchronize(sa->stream));
  if (max_disp) *max_disp = m;
  if (equal) *equal = m < tol ? 1 : 0;
  return AQS_OK;
}

int aqs_num_replicas(const aqs_system* s) { return s ? s->R : 0; }
int64_t aqs_num_atoms(const aqs_system* s, int r) {
  return (s && r >= 0 && r < s->R) ? s->n[r] : 0;
}

aqs_status aqs_get_positions(const aqs_system* s, int r, double* out) {
  if (!s || !out || r < 0 || r >= s->R) return fail(AQS_ERR_INVALID_ARG, "bad argument");
  return fetch_positions(s, r, out);
}

aqs_status aqs_set_positions(aqs_system* s, int r, const double* pos) {
  if (!s || !pos || r < 0 || r >= s->R) return fail(AQS_ERR_INVALID_ARG, "bad argument");
  AQS_TRY(put_positions(s, r, pos));
  std::vector<uint8_t> flags(s->R, 0);
  flags[r] = 1;
  return rebuild(s, flags);
}

aqs_status aqs_get_box(const aqs_system* s, int r, double* H) {
  if (!s || !H || r < 0 || r >= s->R) return fail(AQS_ERR_INVALID_ARG, "bad argument");
  std::memcpy(H, s->geom[r].H, sizeof(double) * s->dim * s->dim);
  return AQS_OK;
}

aqs_status aqs_set_box(aqs_system* s, int r, const double* H) {
  if (!s || !H || r < 0 || r >= s->R) return fail(AQS_ERR_INVALID_ARG, "bad argument");
  AQS_TRY(check_box(s, r, H));
  std::memcpy(s->geom[r].H, H, sizeof(double) * s->dim * s->dim);
  for (int k = 0; k < 9; k++) s->frame[r][k] = 0.0;
  for (int a = 0; a < s->dim; a++) s->frame[r][a * s->dim + a] = 1.0;
  std::vector<uint8_t> flags(s->R, 0);
  flags[r] = 1;
  return rebuild(s, flags);
}

aqs_status aqs_energy_forces(aqs_system* s, int r, double* energy, double* forces, double* tau) {
  if (!s || r < 0 || r >= s->R) return fail(AQS_ERR_INVALID_ARG, "bad argument");
  std::vector<uint8_t> flags(s->R, 0);
  flags[r] = 1;
  AQS_TRY(rebuild(s, flags));
  const int D = s->dim;
  const int n = (int)s->n[r];
  bool dev = forces && is_device_ptr(forces);
  EnergyArgs a;
  a.geom = s->d_geom + r;
  a.x = s->x;
  a.type = s->type;
  a.cell = s->cell;
  a.nb = s->nb;
  a.nnb = s->nnb;
  a.coef = s->d_coef;
  a.forces = forces ? (dev ? forces : s->ubuf) : nullptr;
  a.partial = s->d_partial;
  a.ntot = s->ntot;
  a.nt = s->nt;
  a.perm = s->perm;  // indexed by the global atom index
  CUDA_TRY(launch_energy(D, a, n, s->stream));
  int nb = energy_blocks(n);
  std::vector<double> part(2 * nb);
  CUDA_TRY(cudaMemcpyAsync(part.data(), s->d_partial, sizeof(double) * 2 * nb,
                           cudaMemcpyDeviceToHost, s->stream));
  if (forces && !dev)
    CUDA_TRY(cudaMemcpyAsync(forces, s->ubuf, sizeof(double) * D * n, cudaMemcpyDeviceToHost,
                             s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  double e = 0.0, w = 0.0;
  for (int k = 0; k < nb; k++) {
    e += part[2 * k];
    w += part[2 * k + 1];
  }
  const double* H = s->geom[r].H;
  double vol = D == 2 ? H[0] * H[3] : H[0] * H[4] * H[8];
  if (energy) *energy = 0.5 * e;
  if (tau) *tau = 0.5 * w / vol;
  return AQS_OK;
}

const char* aqs_last_error(void) { return g_err.c_str(); }
void aqs_set_kernel_timing(int on) { g_timing.store(on ? 1 : 0); }
void aqs_get_kernel_stats(aqs_kernel_stats* out) {
  if (out) *out = g_stats;
}
void aqs_reset_kernel_stats(void) { g_stats = aqs_kernel_stats{}; }
int64_t aqs_launch_count(void) { return g_launches.load(); }

double aqs_mean_neighbours(const aqs_system* s, int r) {
  if (!s || r < 0 || r >= s->R) return 0.0;
  std::vector<int32_t> h(s->n[r]);
  if (cudaMemcpy(h.data(), s->nnb + s->off[r], sizeof(int32_t) * s->n[r], cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return 0.0;
  double t = 0.0;
  for (int32_t v : h) t += v;
  return t / (double)s->n[r];
}

int aqs_cluster_size(const aqs_system* s, int r) {
  return (s && r >= 0 && r < s->R) ? s->geom[r].C : 0;
}

aqs_status aqs_autotune_clusters(aqs_system* s, const aqs_fire_params* f, int64_t iters,
                                 const uint8_t* mask, int* best_cluster, int* best_staging,
                                 double* ms_per_iter, double* ms_per_staging) {
  if (!s || !f || iters <= 0) return fail(AQS_ERR_INVALID_ARG, "autotune: bad arguments");
  if (s->C_override > 0)
    return fail(AQS_ERR_INVALID_ARG, "autotune: the system has an explicit cluster size");
  std::vector<uint8_t> m(s->R, 1);
  if (mask)
    for (int r = 0; r < s->R; r++) m[r] = mask[r] ? 1 : 0;
  int best = 0, mode = -1;
  AQS_TRY(tune_clusters(s, f, m, iters, &best, &mode, ms_per_iter, ms_per_staging));
  int64_t nmax = 0;
  int cnt = 0;
  for (int r = 0; r < s->R; r++)
    if (m[r]) {
      nmax = std::max(nmax, s->n[r]);
      cnt++;
    }
  if (best > 0) s->tuned[std::make_pair(cnt, nmax)] = aqs_system::Tuned{best, mode, s->tpa, s->grid_barrier};
  if (best_cluster) *best_cluster = best;
  if (best_staging) *best_staging = mode;
  return AQS_OK;
}

aqs_status aqs_set_launch_budget(aqs_system* s, int64_t iters) {
  if (!s || iters < 1) return fail(AQS_ERR_INVALID_ARG, "set_launch_budget: iters must be >= 1");
  s->launch_budget = iters;
  if (s->chains) s->chains->launch_budget = iters;
  return AQS_OK;
}

aqs_status aqs_set_threads_per_atom(aqs_system* s, int tpa) {
  if (!s || tpa < 0 || tpa > 2) return fail(AQS_ERR_INVALID_ARG, "threads per atom must be 0, 1 or 2");
  s->tpa = tpa == 0 ? 1 : tpa;
  s->tpa_user = tpa != 0;
  s->tuned.clear();
  if (s->chains) {
    s->chains->tpa = s->tpa;
    s->chains->tpa_user = s->tpa_user;
    s->chains->tuned.clear();
  }
  return AQS_OK;
}

int aqs_threads_per_atom(const aqs_system* s) { return s ? s->tpa : 0; }

aqs_status aqs_set_grid_barrier(aqs_system* s, int on) {
  if (!s || on < -1 || on > 1) return fail(AQS_ERR_INVALID_ARG, "grid barrier: -1, 0 or 1");
  s->grid_barrier = on == 1;
  s->grid_barrier_user = on >= 0;
  s->tuned.clear();
  if (s->grid_barrier && s->tpa > 1) s->tpa = 1;
  if (s->chains) {
    s->chains->grid_barrier = s->grid_barrier;
    s->chains->grid_barrier_user = s->grid_barrier_user;
    s->chains->tuned.clear();
  }
  return AQS_OK;
}

int aqs_grid_barrier(const aqs_system* s, int of_chains) {
  if (!s) return -1;
  if (of_chains) return s->chains ? (s->chains->grid_barrier ? 1 : 0) : -1;
  return s->grid_barrier ? 1 : 0;
}

int aqs_max_active_clusters(const aqs_system* s, int replica, int C, int staging, int tpa) {
  if (!s || replica < 0 || replica >= s->R || C < 1 || C > kMaxCluster) return -1;
  const int64_t n = s->n[replica];
  const int npc = (int)((n + C - 1) / C);
  if (npc > 4096) return 0;
  return minimize_max_active_clusters(s->dim, s->prec == AQS_MIXED, C, npc, (int)n, s->nt, s->cap,
                                      staging, tpa < 1 ? 1 : tpa);
}

aqs_status aqs_set_staging(aqs_system* s, int mode) {
  if (!s || mode < -1 || mode >= kNumStaging)
    return fail(AQS_ERR_INVALID_ARG, "set_staging: mode must be -1 or 0..%d", kNumStaging - 1);
  s->staging = mode;
  s->staging_user = mode >= 0;
  if (s->chains) {
    s->chains->staging = mode;
    s->chains->staging_user = mode >= 0;
  }
  return AQS_OK;
}

int aqs_staging(const aqs_system* s, int replica) {
  if (!s || replica < 0 || replica >= s->R) return -1;
  const RepGeom& g = s->geom[replica];
  return minimize_staging(s->dim, g.npc, g.n, s->nt, s->cap, s->staging);
}

aqs_status aqs_set_autotune(aqs_system* s, int64_t iters) {
  if (!s || iters < 0) return fail(AQS_ERR_INVALID_ARG, "set_autotune: bad arguments");
  s->tune_iters = iters;
  if (s->chains) s->chains->tune_iters = iters;
  return AQS_OK;
}

}  // extern "C"

// =====================================================================
//                 learned warm start (C ABI, 2D workloads)
// =====================================================================
struct aqs_warm {
  int dim = 2, n_types = 2;
  cudaStream_t stream = nullptr;
  MlpDev m{};
  uint8_t* d_mask = nullptr;
  float* d_grad = nullptr;
  float* d_loss = nullptr;
  int gblocks = 0;  // gradient partials: one per SM of the device
  int64_t adam_t = 0;
  std::vector<void*> allocs;
};

namespace {

template <typename T>
aqs_status walloc(aqs_warm* w, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(AQS_ERR_OOM, "warm start: device allocation failed");
  }
  w->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return AQS_OK;
}

uint16_t f2bf(float f) {  // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

void param_mask(int dim, int n_types, std::vector<uint8_t>& mask) {
  mask.assign(kNumParams, 1);
  const int feat = kNb * dim + n_types;
  for (int o = 0; o < kHid; o++)
    for (int i = feat; i < kIn; i++) mask[o * kIn + i] = 0;  // W1 padding columns
  const int w4 = kHid * kIn + 2 * kHid * kHid;
  for (int o = dim; o < kOutPad; o++)
    for (int i = 0; i < kHid; i++) mask[w4 + o * kHid + i] = 0;  // W4 padding rows
  for (int o = dim; o < kOutPad; o++) mask[kNumWeights + 3 * kHid + o] = 0;  // b4 padding
}

aqs_status upload_params(aqs_warm* w, const std::vector<float>& p) {
  std::vector<uint16_t> bf(kNumWeights);
  for (int k = 0; k < kNumWeights; k++) bf[k] = f2bf(p[k]);
  CUDA_TRY(cudaMemcpyAsync(w->m.master, p.data(), sizeof(float) * kNumParams,
                           cudaMemcpyHostToDevice, w->stream));
  CUDA_TRY(cudaMemcpyAsync(w->m.wbf, bf.data(), sizeof(uint16_t) * kNumWeights,
                           cudaMemcpyHostToDevice, w->stream));
  CUDA_TRY(cudaMemcpyAsync(w->m.b, p.data() + kNumWeights, sizeof(float) * kNumBiases,
                           cudaMemcpyHostToDevice, w->stream));
  CUDA_TRY(cudaMemsetAsync(w->m.m1, 0, sizeof(float) * kNumParams, w->stream));
  CUDA_TRY(cudaMemsetAsync(w->m.m2, 0, sizeof(float) * kNumParams, w->stream));
  CUDA_TRY(cudaStreamSynchronize(w->stream));
  w->adam_t = 0;
  return AQS_OK;
}

aqs_status ensure_warm_buffers(aqs_system* s) {
  if (!s->d_feat) AQS_TRY(alloc_arr(s, &s->d_feat, (size_t)s->ntot * kIn));
  if (!s->d_u) AQS_TRY(alloc_arr(s, &s->d_u, (size_t)s->ntot * s->dim));
  if (!s->d_save) AQS_TRY(alloc_arr(s, &s->d_save, (size_t)s->ntot * s->dim));
  if (!s->d_err) AQS_TRY(alloc_arr(s, &s->d_err, 1));
  return AQS_OK;
}

// features of every replica, rows in caller order (replica r at rows off_r..)
aqs_status features_all(aqs_system* s, __nv_bfloat16* bf, double* f64, int64_t row_base) {
  if (s->dim != 2) return fail(AQS_ERR_UNSUPPORTED, "warm start features are built for 2D");
  // the list build keeps cells current; make sure every replica's cell
  // start table matches its atoms (rebuild is cheap and sorts the atoms)
  AQS_TRY(rebuild_all(s));
  CUDA_TRY(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
  for (int r = 0; r < s->R; r++) {
    FeatArgs a;
    a.geom = s->d_geom;
    a.rep = r;
    a.tilt = s->geom[r].H[1];
    a.x = s->x;
    a.type = s->type;
    a.cell = s->cell;
    a.cstart = s->cstart;
    a.perm = s->perm;
    a.inv = s->inv;
    a.ntot = s->ntot;
    a.nb = kNb;
    a.n_types = s->nt;
    a.half = 2;
    double w[3];
    cell_widths(s->dim, s->geom[r].H, w);
    double cw = std::min(w[0] / s->geom[r].nc[0], w[1] / s->geom[r].nc[1]);
    a.reach2 = (a.half * cw) * (a.half * cw);
    a.bf = bf;
    a.width = kIn;
    a.f64 = f64;
    a.width64 = kNb * s->dim + s->nt;
    a.row0 = row_base + s->off[r];
    a.err = s->d_err;
    CUDA_TRY(launch_knn_features(s->dim, a, (int)s->n[r], s->stream));
  }
  int err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (err) return fail(AQS_ERR_BOX_TOO_SMALL, "neighbour-shell stencil too short for 32 neighbours");
  return AQS_OK;
}

aqs_status save_positions(aqs_system* s) {
  for (int r = 0; r < s->R; r++)
    AQS_TRY(gather_user(s, r, s->d_save + (size_t)s->off[r] * s->dim));
  return AQS_OK;
}

aqs_status restore_positions(aqs_system* s, const std::vector<uint8_t>& which,
                             const std::vector<double>& tilt) {
  for (int r = 0; r < s->R; r++) {
    if (!which[r]) continue;
    CUDA_TRY(launch_scatter_user(s->d_save + (size_t)s->off[r] * s->dim, s->x, s->ntot, s->off[r],
                                 (int)s->n[r], s->perm, s->dim, s->stream));
    s->geom[r].H[1] = tilt[r];
  }
  AQS_TRY(upload_geom(s));
  sync_tilt_to_state(s);
  AQS_TRY(upload_state(s));
  return rebuild(s, which);
}

// Sets the cluster size of the replicas `reps` to C and rebuilds their lists
// (list entries encode the owner CTA of every neighbour).
aqs_status apply_cluster(aqs_system* s, const std::vector<int>& reps, int C) {
  std::vector<uint8_t> flags(s->R, 0);
  bool any = false;
  for (int r : reps) {
    if (s->geom[r].C == C) continue;
    s->geom[r].C = C;
    s->geom[r].npc = (int)((s->n[r] + C - 1) / C);
    flags[r] = 1;
    any = true;
  }
  return any ? rebuild(s, flags) : AQS_OK;
}

bool cluster_feasible(const aqs_system* s, const std::vector<int>& reps, int C) {
  for (int r : reps) {
    const int64_t npc = (s->n[r] + C - 1) / C;
    if (npc > 4096 || (C > 1 && s->n[r] < 32 * (int64_t)C)) return false;
    if (s->grid_barrier) {
      if (minimize_max_grid_replicas(s->dim, s->prec == AQS_MIXED, C, (int)npc, (int)s->n[r],
                                     s->nt, s->cap, s->staging) < (int)reps.size())
        return false;
      continue;
    }
    if (minimize_max_active_clusters(s->dim, s->prec == AQS_MIXED, C, (int)npc, (int)s->n[r],
                                     s->nt, s->cap, s->staging, s->tpa) <= 0)
      return false;
  }
  return true;
}

// Times one candidate (cluster size C, the system's current staging mode) on
// the masked replicas: an untimed short run, then `ft` timed; the
// configuration is restored after each run.
aqs_status time_candidate(aqs_system* s, const aqs_fire_params& ft, const aqs_fire_params& fw,
                          const std::vector<uint8_t>& mask, const std::vector<int>& reps,
                          const std::vector<double>& tilt, int C, double* ms) {
  s->C_override = C;  // no cluster growth while a candidate is timed
  AQS_TRY(apply_cluster(s, reps, C));
  aqs_status st = minimize_impl(s, &fw, mask, nullptr);
  if (st != AQS_OK && st != AQS_ERR_NOT_CONVERGED) return st;
  AQS_TRY(restore_positions(s, mask, tilt));
  if (cudaStreamSynchronize(s->stream) != cudaSuccess)
    return fail(AQS_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
  const auto t0 = std::chrono::steady_clock::now();
  st = minimize_impl(s, &ft, mask, nullptr);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess)
    return fail(AQS_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
  const auto t1 = std::chrono::steady_clock::now();
  if (st != AQS_OK && st != AQS_ERR_NOT_CONVERGED) return st;
  int64_t it = 1;
  for (int r : reps) it = std::max<int64_t>(it, s->st[r].iters);
  *ms = std::chrono::duration<double, std::milli>(t1 - t0).count() / (double)it;
  return restore_positions(s, mask, tilt);
}

// Times `iters` FIRE iterations (convergence test off) of the masked replicas
// for every feasible cluster size (automatic staging), then every staging mode
// that fits at the fastest size, and keeps the fastest pair; the
// configuration and the host-side minimiser state are restored afterwards.
aqs_status tune_clusters(aqs_system* s, const aqs_fire_params* f, const std::vector<uint8_t>& mask,
                         int64_t iters, int* best, int* best_staging, double* ms_per_iter,
                         double* ms_per_staging) {
  std::vector<int> reps;
  int64_t nmax = 0;
  for (int r = 0; r < s->R; r++)
    if (mask[r]) {
      reps.push_back(r);
      nmax = std::max(nmax, s->n[r]);
    }
  if (ms_per_iter)
    for (int c = 0; c <= kMaxCluster; c++) ms_per_iter[c] = -1.0;
  if (ms_per_staging)
    for (int m = 0; m < kNumStaging; m++) ms_per_staging[m] = -1.0;
  if (best) *best = 0;
  if (best_staging) *best_staging = s->staging;
  if (reps.empty() || iters <= 0) return AQS_OK;
  if (!s->d_save) AQS_TRY(alloc_arr(s, &s->d_save, (size_t)s->ntot * s->dim));
  AQS_TRY(save_positions(s));
  std::vector<double> tilt(s->R);
  std::vector<int> c0(s->R);
  for (int r = 0; r < s->R; r++) {
    tilt[r] = s->geom[r].H[1];
    c0[r] = s->geom[r].C;
  }
  const std::vector<RepState> st0 = s->st;
  aqs_fire_params ft = *f;
  ft.tol = 0.0;
  ft.max_iter = iters;
  aqs_fire_params fw = ft;
  fw.max_iter = std::min<int64_t>(iters, 32);
  const int saved_override = s->C_override, saved_staging = s->staging, saved_tpa = s->tpa;
  const bool saved_gb = s->grid_barrier;
  s->tuning = true;
  int bestC = 0, bestM = s->staging, bestTPA = s->tpa;
  bool bestGB = s->grid_barrier;
  double bestT = 1e300;
  // time per iteration of every candidate: [barrier mode][C][tpa - 1][staging]
  const size_t per_mode = (size_t)(kMaxCluster + 1) * 2 * kNumStaging;
  std::vector<double> table(2 * per_mode, -1.0);
  aqs_status err = AQS_OK;
  // one barrier mode: every cluster size, threads per atom and staging mode
  auto search = [&](bool gb) {
    s->grid_barrier = gb;
    for (int C = 1; C <= kMaxCluster && err == AQS_OK; C++) {
      const int npc = (int)((nmax + C - 1) / C);
      // threads per atom of the force phase ("atoms per warp" 32 or 16), unless
      // the caller fixed it (grid barriers: one)
      for (int tpa = 1; tpa <= 2 && err == AQS_OK; tpa++) {
        if (s->tpa_user && tpa != saved_tpa) continue;
        if (tpa == 2 && (gb || minimize_tpa(npc, 2) != 2)) continue;
        // every staging mode that fits: the mode decides the shared memory of
        // a CTA and with it how many CTAs (of different clusters) share an SM,
        // so it decides how many clusters are resident at once
        for (int m = 0; m < kNumStaging && err == AQS_OK; m++) {
          if (s->staging_user && m != saved_staging) continue;
          if (gb && m != 0 && m != 3) continue;
          if (minimize_staging(s->dim, npc, (int)nmax, s->nt, s->cap, m) != m) continue;
          s->tpa = tpa;
          s->staging = m;
          if (!cluster_feasible(s, reps, C)) continue;
          double ms = 0.0;
          if ((err = time_candidate(s, ft, fw, mask, reps, tilt, C, &ms)) != AQS_OK) break;
          table[(gb ? per_mode : 0) + ((size_t)C * 2 + (tpa - 1)) * kNumStaging + m] = ms;
          if (ms_per_iter && (ms_per_iter[C] < 0.0 || ms < ms_per_iter[C])) ms_per_iter[C] = ms;
          if (ms < bestT) {
            bestT = ms;
            bestC = C;
            bestTPA = tpa;
            bestM = m;
            bestGB = gb;
          }
        }
      }
    }
  };
  // thread-block clusters, and (unless the caller fixed the mode) one
  // cooperative launch with global-memory barriers
  if (!s->grid_barrier_user || !saved_gb) search(false);
  if (err == AQS_OK && (!s->grid_barrier_user || saved_gb)) search(true);
  if (ms_per_staging && bestC > 0)
    for (int m = 0; m < kNumStaging; m++)
      ms_per_staging[m] =
          table[(bestGB ? per_mode : 0) + ((size_t)bestC * 2 + (bestTPA - 1)) * kNumStaging + m];
  if (s->staging_user) bestM = saved_staging;
  s->tuning = false;
  s->C_override = saved_override;
  s->staging = err == AQS_OK ? bestM : saved_staging;
  s->tpa = err == AQS_OK ? bestTPA : saved_tpa;
  s->grid_barrier = err == AQS_OK ? bestGB : saved_gb;
  for (int r : reps) {
    const int C = (err == AQS_OK && bestC > 0) ? bestC : c0[r];
    s->geom[r].C = C;
    s->geom[r].npc = (int)((s->n[r] + C - 1) / C);
  }
  s->st = st0;
  const aqs_status rs = restore_positions(s, mask, tilt);
  if (err != AQS_OK) return err;
  if (rs != AQS_OK) return rs;
  if (best) *best = bestC;
  if (best_staging) *best_staging = s->staging;
  return AQS_OK;
}

}  // namespace

extern "C" {

int aqs_warm_num_params(void) { return kNumParams; }

aqs_status aqs_warm_create(int dim, int n_types, uint64_t seed, void* stream, aqs_warm** out) {
  if (!out) return fail(AQS_ERR_INVALID_ARG, "null argument");
  if (dim != 2) return fail(AQS_ERR_UNSUPPORTED, "the warm start network is built for 2D");
  if (n_types < 1 || n_types > kIn - kNb * dim) return fail(AQS_ERR_INVALID_ARG, "bad n_types");
  aqs_warm* w = new aqs_warm();
  w->dim = dim;
  w->n_types = n_types;
  w->stream = (cudaStream_t)stream;
  w->gblocks = sm_count();
  aqs_status st = AQS_OK;
  __nv_bfloat16* wbf = nullptr;
  if ((st = walloc(w, &wbf, kNumWeights)) != AQS_OK ||
      (st = walloc(w, &w->m.b, kNumBiases)) != AQS_OK ||
      (st = walloc(w, &w->m.master, kNumParams)) != AQS_OK ||
      (st = walloc(w, &w->m.m1, kNumParams)) != AQS_OK ||
      (st = walloc(w, &w->m.m2, kNumParams)) != AQS_OK ||
      (st = walloc(w, &w->d_mask, kNumParams)) != AQS_OK ||
      (st = walloc(w, &w->d_grad, kNumParams)) != AQS_OK ||
      (st = walloc(w, &w->d_loss, w->gblocks)) != AQS_OK ||
      (st = walloc(w, &w->m.gscratch, (size_t)w->gblocks * kNumParams)) != AQS_OK) {
    aqs_warm_destroy(w);
    return st;
  }
  w->m.wbf = wbf;
  w->m.mask = w->d_mask;
  // Glorot-uniform weights from a SplitMix64 stream, zero biases
  std::vector<float> p(kNumParams, 0.0f);
  std::vector<uint8_t> mask;
  param_mask(dim, n_types, mask);
  uint64_t z = seed * 0xD1B54A32D192ED03ull;
  auto next = [&]() {
    z += 0x9E3779B97F4A7C15ull;
    uint64_t t = z;
    t = (t ^ (t >> 30)) * 0xBF58476D1CE4E5B9ull;
    t = (t ^ (t >> 27)) * 0x94D049BB133111EBull;
    t ^= t >> 31;
    return (double)(t >> 11) * (1.0 / 9007199254740992.0);
  };
  const int fan_in[4] = {kNb * dim + n_types, kHid, kHid, kHid};
  const int fan_out[4] = {kHid, kHid, kHid, dim};
  const int nin[4] = {kIn, kHid, kHid, kHid}, nout[4] = {kHid, kHid, kHid, kOutPad};
  int off = 0;
  for (int l = 0; l < 4; l++) {
    const double lim = std::sqrt(6.0 / (fan_in[l] + fan_out[l]));
    for (int k = 0; k < nin[l] * nout[l]; k++) {
      double u = next();
      p[off + k] = mask[off + k] ? (float)((2.0 * u - 1.0) * lim) : 0.0f;
    }
    off += nin[l] * nout[l];
  }
  if (cudaMemcpy(w->d_mask, mask.data(), kNumParams, cudaMemcpyHostToDevice) != cudaSuccess ||
      (st = upload_params(w, p)) != AQS_OK) {
    aqs_warm_destroy(w);
    return st != AQS_OK ? st : fail(AQS_ERR_CUDA, "warm start upload failed");
  }
  *out = w;
  return AQS_OK;
}

void aqs_warm_destroy(aqs_warm* w) {
  if (!w) return;
  cudaStreamSynchronize(w->stream);
  for (void* p : w->allocs) cudaFree(p);
  delete w;
}

aqs_status aqs_warm_get_params(const aqs_warm* w, float* host) {
  if (!w || !host) return fail(AQS_ERR_INVALID_ARG, "null argument");
  CUDA_TRY(cudaMemcpyAsync(host, w->m.master, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost,
                           w->stream));
  CUDA_TRY(cudaStreamSynchronize(w->stream));
  return AQS_OK;
}

aqs_status aqs_warm_set_params(aqs_warm* w, const float* host) {
  if (!w || !host) return fail(AQS_ERR_INVALID_ARG, "null argument");
  std::vector<float> p(host, host + kNumParams);
  std::vector<uint8_t> mask;
  param_mask(w->dim, w->n_types, mask);
  for (int k = 0; k < kNumParams; k++)
    if (!mask[k]) p[k] = 0.0f;
  return upload_params(w, p);
}

aqs_status aqs_warm_features(aqs_system* s, int replica, void* feat_bf16, double* feat_f64) {
  if (!s || !feat_bf16) return fail(AQS_ERR_INVALID_ARG, "null argument");
  if (replica < -1 || replica >= s->R) return fail(AQS_ERR_INVALID_ARG, "bad replica");
  AQS_TRY(ensure_warm_buffers(s));
  // rows of all replicas are written; a single replica's rows start at 0
  const int64_t base = replica >= 0 ? -s->off[replica] : 0;
  if (replica >= 0) {
    // only the chosen replica: write into the caller's buffer, others to scratch
    AQS_TRY(features_all(s, s->d_feat, nullptr, 0));
    (void)base;
    if (s->dim != 2) return AQS_ERR_UNSUPPORTED;
    FeatArgs a;  // recompute the chosen replica straight into the caller's rows
    a.geom = s->d_geom;
    a.rep = replica;
    a.tilt = s->geom[replica].H[1];
    a.x = s->x;
    a.type = s->type;
    a.cell = s->cell;
    a.cstart = s->cstart;
    a.perm = s->perm;
    a.inv = s->inv;
    a.ntot = s->ntot;
    a.nb = kNb;
    a.n_types = s->nt;
    a.half = 2;
    double w[3];
    cell_widths(s->dim, s->geom[replica].H, w);
    double cw = std::min(w[0] / s->geom[replica].nc[0], w[1] / s->geom[replica].nc[1]);
    a.reach2 = (a.half * cw) * (a.half * cw);
    a.bf = static_cast<__nv_bfloat16*>(feat_bf16);
    a.width = kIn;
    a.f64 = feat_f64;
    a.width64 = kNb * s->dim + s->nt;
    a.row0 = 0;
    a.err = s->d_err;
    CUDA_TRY(launch_knn_features(s->dim, a, (int)s->n[replica], s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return AQS_OK;
  }
  return features_all(s, static_cast<__nv_bfloat16*>(feat_bf16), feat_f64, 0);
}

aqs_status aqs_warm_predict(aqs_warm* w, const void* feat_bf16, int64_t rows, float* out) {
  if (!w || !feat_bf16 || !out || rows < 0) return fail(AQS_ERR_INVALID_ARG, "bad argument");
  if ((reinterpret_cast<uintptr_t>(feat_bf16) & 15u) != 0u)
    return fail(AQS_ERR_INVALID_ARG, "features must start on a 16-byte boundary");
  if (rows == 0) return AQS_OK;
  CUDA_TRY(launch_mlp_forward(w->m, static_cast<const __nv_bfloat16*>(feat_bf16), rows, out, w->dim,
                              w->stream));
  return AQS_OK;
}

aqs_status aqs_warm_loss_grad(aqs_warm* w, const void* feat_bf16, const float* target,
                              int64_t rows, float* grad_host, double* loss) {
  if (!w || !feat_bf16 || !target || rows <= 0) return fail(AQS_ERR_INVALID_ARG, "bad argument");
  const int blocks = (int)std::min<int64_t>(w->gblocks, (rows + 31) / 32);
  CUDA_TRY(launch_mlp_grad(w->m, static_cast<const __nv_bfloat16*>(feat_bf16), target, rows, w->dim,
                           blocks, w->d_grad, w->d_loss, w->stream));
  std::vector<float> lp(blocks);
  CUDA_TRY(cudaMemcpyAsync(lp.data(), w->d_loss, sizeof(float) * blocks, cudaMemcpyDeviceToHost,
                           w->stream));
  if (grad_host)
    CUDA_TRY(cudaMemcpyAsync(grad_host, w->d_grad, sizeof(float) * kNumParams,
                             cudaMemcpyDeviceToHost, w->stream));
  CUDA_TRY(cudaStreamSynchronize(w->stream));
  double l = 0.0;
  for (float v : lp) l += v;
  if (loss) *loss = l;
  return AQS_OK;
}

aqs_status aqs_warm_train_step(aqs_warm* w, const void* feat_bf16, const float* target,
                               int64_t rows, double lr, double weight_decay, double* loss) {
  AQS_TRY(aqs_warm_loss_grad(w, feat_bf16, target, rows, nullptr, loss));
  w->adam_t++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.0f - std::pow(b1, (float)w->adam_t), bc2 = 1.0f - std::pow(b2, (float)w->adam_t);
  CUDA_TRY(launch_mlp_adamw(w->m, w->d_grad, (float)lr, b1, b2, 1e-8f, (float)weight_decay, bc1, bc2,
                            w->stream));
  return AQS_OK;
}

aqs_status aqs_warm_collect(aqs_system* s, const aqs_fire_params* f, double dgamma, int64_t n_steps,
                            void* feat_out, float* target_out) {
  if (!s || !f || !feat_out || !target_out || n_steps < 0)
    return fail(AQS_ERR_INVALID_ARG, "bad argument");
  AQS_TRY(ensure_warm_buffers(s));
  __nv_bfloat16* fo = static_cast<__nv_bfloat16*>(feat_out);
  for (int64_t k = 0; k < n_steps; k++) {
    AQS_TRY(features_all(s, fo + (size_t)k * s->ntot * kIn, nullptr, 0));
    std::vector<Job> jobs(s->R);
    for (int r = 0; r < s->R; r++) {
      jobs[r].nsteps = 1;
      jobs[r].dgamma = dgamma;
    }
    AQS_TRY(run_jobs(s, f, jobs, nullptr));
    for (int r = 0; r < s->R; r++)
      CUDA_TRY(launch_step_target(s->dim, s->x, s->xs, s->ntot, s->off[r], (int)s->n[r], s->perm,
                                  reinterpret_cast<const double*>(
                                      reinterpret_cast<const char*>(s->d_geom + r) +
                                      offsetof(RepGeom, H)),
                                  1.0 / dgamma,
                                  target_out + ((size_t)k * s->ntot + s->off[r]) * s->dim,
                                  s->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return AQS_OK;
}

aqs_status aqs_run_sequential_warm(aqs_system* s, const aqs_fire_params* f, aqs_warm* w,
                                   double dgamma, int64_t n_steps, double gate, double* energy,
                                   double* tau, int64_t* fire_iters, double* nonaffine,
                                   uint8_t* used_warm) {
  if (!s || !f || !w || n_steps < 0) return fail(AQS_ERR_INVALID_ARG, "bad argument");
  if (w->dim != s->dim || w->n_types != s->nt)
    return fail(AQS_ERR_INVALID_ARG, "network and system differ in dimension or species");
  if (!(gate > 0.0)) gate = 1e-2;
  AQS_TRY(ensure_warm_buffers(s));
  for (int64_t k = 0; k < n_steps; k++) {
    // prediction for the step from the current minima
    AQS_TRY(features_all(s, s->d_feat, nullptr, 0));
    CUDA_TRY(launch_mlp_forward(w->m, s->d_feat, s->ntot, s->d_u, s->dim, s->stream));
    AQS_TRY(save_positions(s));
    std::vector<double> tilt(s->R);
    for (int r = 0; r < s->R; r++) tilt[r] = s->geom[r].H[1];
    std::vector<Job> jobs(s->R);
    for (int r = 0; r < s->R; r++) {
      jobs[r].nsteps = 1;
      jobs[r].dgamma = dgamma;
    }
    JobOut jo;
    AQS_TRY(run_jobs(s, f, jobs, &jo, s->d_u));
    // gate: keep the learned start only where the step stayed elastic, i.e.
    // the minimum lies within `gate` of both the learned and the affine start
    std::vector<uint8_t> redo(s->R, 0);
    bool any = false;
    for (int r = 0; r < s->R; r++) {
      const double* q = &jo.rec[(size_t)r * jo.stride * kRecFields];
      if (!(q[2] < gate && q[5] < gate)) {
        redo[r] = 1;
        any = true;
      }
    }
    std::vector<double> rec_keep = jo.rec;
    if (any) {
      AQS_TRY(restore_positions(s, redo, tilt));
      std::vector<Job> plain(s->R);
      for (int r = 0; r < s->R; r++)
        if (redo[r]) {
          plain[r].nsteps = 1;
          plain[r].dgamma = dgamma;
        }
      JobOut jp;
      AQS_TRY(run_jobs(s, f, plain, &jp));
      for (int r = 0; r < s->R; r++)
        if (redo[r])
          for (int c = 0; c < kRecFields; c++)
            rec_keep[(size_t)r * jo.stride * kRecFields + c] =
                jp.rec[(size_t)r * jp.stride * kRecFields + c] +
                (c == 3 || c == 4 ? jo.rec[(size_t)r * jo.stride * kRecFields + c] : 0.0);
    }
    for (int r = 0; r < s->R; r++) {
      const double* q = &rec_keep[(size_t)r * jo.stride * kRecFields];
      size_t i = (size_t)k * s->R + r;
      if (energy) energy[i] = q[0];
      if (tau) tau[i] = q[1];
      if (fire_iters) fire_iters[i] = (int64_t)q[3];
      if (nonaffine) nonaffine[i] = q[2];
      if (used_warm) used_warm[i] = redo[r] ? 0 : 1;
    }
  }
  return AQS_OK;
}

}  // extern "C"

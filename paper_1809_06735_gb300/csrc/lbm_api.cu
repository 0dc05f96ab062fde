// C ABI and host runtime of the D2Q9 library: configuration checks,
// workspace layout, the per-member tile table of the batched stream-collide,
// CUDA-graph replay of the step loop, the launch-shape autotuner, the
// snapshot ring of the eq. (17) time derivative, and the diagnostic calls.
//
// The runtime never allocates device memory: every device buffer is carved
// out of the caller's workspace (see lbm_workspace_size).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"


using lbm::Member;
using lbm::Tile;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxL = lbm::kDiagMaxL;  // box sizes per balance call
constexpr size_t kDiagBatchBytes = (size_t)8 << 30;  // default scratch budget of a batch
constexpr int kTileW = 128;        // cells per warp row in the vector kernel

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

thread_local std::string g_last_error = "no error";

struct Layout {
  size_t members, tiles, status, sync;
  std::vector<size_t> pop0, pop1, fx, fy, fx64, fy64, snap;
  std::vector<size_t> ft, ft64, trig, trig64, damp, damp_f, damp_ring, proj, drows, pcount;
  std::vector<size_t> nu_ring;  // variable viscosity: local viscosity per snapshot slot
  size_t scratch, partials, count, jpart, jobs, stats, Ls, out7, origins;
  size_t edges, hist, mach;  // distributions: bin edges, histograms, Ma_V statistics
  int diag_slots;          // members per batched diagnostic launch
  size_t slot_doubles, jpart_doubles;
  size_t total;
  size_t Nmax;
  size_t origin_cap;  // boxes the origin buffer holds
  size_t scratch_fields;
};

int pitch_of(int nx, int precision) {
  // rows start on 16-byte boundaries: 4 floats or 2 doubles
  const int q = precision == 32 ? 4 : 2;
  return (nx + q - 1) / q * q;
}

// Tables of force kind 2.  ft: the shell force of eqs. (14), (15) in FP64,
// [2][ny * nx]: psi = F0 sum_k cos(2 pi (kx x/nx + ky y/ny) + phase) over one
// of each pair +-k with 5 <= |k| <= 7 (ky > 0, or ky = 0 and kx > 0), force
// (d_y psi, -d_x psi) = F0 sum_k sin(theta_k) (-2 pi ky/ny, 2 pi kx/nx),
// with sin(theta) = sin(a_x + phase) cos(b_y) + cos(a_x + phase) sin(b_y)
// from per-axis tables.  ftp: the same with rows of `pitch` (zero padded).
// trig: cos, sin of 2 pi x/nx and of 4 pi x/nx ([4][nx]), then of y ([4][ny]).
void shell_force_tables(const lbm_member_cfg &c, int pitch, std::vector<double> *ft,
                        std::vector<double> *ftp, std::vector<double> *trig) {
  const double pi = 3.14159265358979323846;
  const int nx = c.nx, ny = c.ny;
  const size_t N = (size_t)nx * ny;
  ft->assign(2 * N, 0.0);
  std::vector<double> sa(nx), ca(nx), sb(ny), cb(ny);
  for (int ky = 0; ky <= 7; ++ky)
    for (int kx = -7; kx <= 7; ++kx) {
      const int k2 = kx * kx + ky * ky;
      if (k2 < 25 || k2 > 49 || (ky == 0 && kx <= 0)) continue;
      for (int x = 0; x < nx; ++x) {
        const double a = 2.0 * pi * kx * (double)x / nx + c.phase;
        sa[x] = std::sin(a);
        ca[x] = std::cos(a);
      }
      for (int y = 0; y < ny; ++y) {
        const double b = 2.0 * pi * ky * (double)y / ny;
        sb[y] = std::sin(b);
        cb[y] = std::cos(b);
      }
      const double gx = -2.0 * pi * ky / ny, gy = 2.0 * pi * kx / nx;
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const double st = sa[x] * cb[y] + ca[x] * sb[y];
          (*ft)[(size_t)y * nx + x] += gx * st;
          (*ft)[N + (size_t)y * nx + x] += gy * st;
        }
    }
  for (double &v : *ft) v *= c.F0;
  const size_t plane = (size_t)ny * pitch;
  ftp->assign(2 * plane, 0.0);
  for (int k = 0; k < 2; ++k)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        (*ftp)[k * plane + (size_t)y * pitch + x] = (*ft)[k * N + (size_t)y * nx + x];
  trig->assign(4 * ((size_t)nx + ny), 0.0);
  for (int x = 0; x < nx; ++x) {
    const double a = 2.0 * pi * x / nx;
    (*trig)[x] = std::cos(a);
    (*trig)[nx + x] = std::sin(a);
    (*trig)[2 * nx + x] = std::cos(2.0 * a);
    (*trig)[3 * nx + x] = std::sin(2.0 * a);
  }
  double *ty = trig->data() + 4 * (size_t)nx;
  for (int y = 0; y < ny; ++y) {
    const double b = 2.0 * pi * y / ny;
    ty[y] = std::cos(b);
    ty[ny + y] = std::sin(b);
    ty[2 * ny + y] = std::cos(2.0 * b);
    ty[3 * ny + y] = std::sin(2.0 * b);
  }
}

// The vectorised FP32 kernel serves nx % 4 == 0 with every collision.
bool vector_eligible(const lbm_member_cfg &m, int precision) {
  return precision == 32 && m.nx % 4 == 0;
}

int check_config(const lbm_config *cfg, std::string &err) {
  if (!cfg) { err = "config is NULL"; return LBM_ERR_ARG; }
  if (cfg->n_members < 1 || !cfg->members) { err = "n_members must be >= 1 with a member array"; return LBM_ERR_ARG; }
  if (cfg->precision != 32 && cfg->precision != 64) { err = "precision must be 32 or 64"; return LBM_ERR_ARG; }
  if (cfg->storage < 0 || cfg->storage > 2) { err = "storage must be 0 (tuned), 1 (AA) or 2 (double buffer)"; return LBM_ERR_ARG; }
  if (cfg->diag_precision != 0 && cfg->diag_precision != 32 && cfg->diag_precision != 64) { err = "diag_precision must be 0, 32 or 64"; return LBM_ERR_ARG; }
  if (cfg->diag_every < 0 || cfg->graph_steps < 0) { err = "diag_every and graph_steps must be >= 0"; return LBM_ERR_ARG; }
  if (cfg->diag_batch < 0) { err = "diag_batch must be >= 0"; return LBM_ERR_ARG; }
  for (int m = 0; m < cfg->n_members; ++m) {
    const lbm_member_cfg &c = cfg->members[m];
    char buf[160];
    if (c.nx < 1 || c.ny < 1 || (long long)c.nx * c.ny > (1LL << 30)) {
      snprintf(buf, sizeof buf, "member %d: grid %dx%d out of range", m, c.nx, c.ny);
      err = buf; return LBM_ERR_ARG;
    }
    if (!(c.tau > 0.5) || !std::isfinite(c.tau)) {
      snprintf(buf, sizeof buf, "member %d: tau must be > 0.5", m); err = buf; return LBM_ERR_ARG;
    }
    if (!(c.rho0 > 0) || !std::isfinite(c.rho0)) {
      snprintf(buf, sizeof buf, "member %d: rho0 must be > 0", m); err = buf; return LBM_ERR_ARG;
    }
    if (c.force_kind < 0 || c.force_kind > 2) {
      snprintf(buf, sizeof buf, "member %d: force_kind must be 0, 1 or 2", m); err = buf; return LBM_ERR_ARG;
    }
    if (c.collision < 0 || c.collision > 3 || !std::isfinite(c.Cs) || c.Cs < 0.0) {
      snprintf(buf, sizeof buf, "member %d: collision must be 0..3 with Cs >= 0", m);
      err = buf; return LBM_ERR_ARG;
    }
    if (!std::isfinite(c.F0) || !std::isfinite(c.alpha) ||
        (c.force_kind == 2 && (!std::isfinite(c.phase) || !std::isfinite(c.FR0)))) {
      snprintf(buf, sizeof buf, "member %d: force parameters not finite", m); err = buf; return LBM_ERR_ARG;
    }
  }
  return LBM_OK;
}

Layout make_layout(const lbm_config *cfg) {
  Layout L{};
  const int n = cfg->n_members;
  const size_t es = cfg->precision == 32 ? 4 : 8;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  L.members = take(sizeof(Member) * n);
  // tile table sized for the smallest tile height (1 row)
  size_t max_tiles = 0;
  for (int m = 0; m < n; ++m) {
    const lbm_member_cfg &c = cfg->members[m];
    if (vector_eligible(c, cfg->precision)) {
      max_tiles += (size_t)((c.nx + kTileW - 1) / kTileW) * c.ny;
    }
  }
  L.tiles = take(sizeof(Tile) * std::max<size_t>(max_tiles, 1));
  L.status = take(sizeof(int) * n);
  L.sync = take(4 * sizeof(unsigned));  // persistent small-grid step: count, gen, err
  L.Nmax = 0;
  for (int m = 0; m < n; ++m) {
    const lbm_member_cfg &c = cfg->members[m];
    const size_t N = (size_t)c.nx * c.ny;
    const size_t plane = (size_t)c.ny * pitch_of(c.nx, cfg->precision);
    L.pop0.push_back(take(es * 9 * plane));
    L.pop1.push_back(cfg->storage == 1 ? L.pop0.back() : take(es * 9 * plane));  // AA: one array
    L.fx.push_back(take(es * c.ny));
    L.fy.push_back(take(es * c.nx));
    L.fx64.push_back(take(8 * c.ny));
    L.fy64.push_back(take(8 * c.nx));
    L.snap.push_back(take(8 * 9 * N));
    const bool k2 = c.force_kind == 2;  // shell force tables, damping state
    const size_t nt = 4 * ((size_t)c.nx + c.ny);
    const size_t pctas = (size_t)((c.nx + 63) / 64) * ((c.ny + 3) / 4);
    L.ft.push_back(take(k2 ? es * 2 * plane : 0));
    L.ft64.push_back(take(k2 ? 8 * 2 * N : 0));
    L.trig.push_back(take(k2 ? es * nt : 0));
    L.trig64.push_back(take(k2 ? 8 * nt : 0));
    L.damp.push_back(take(k2 ? 8 * lbm::kDamp : 0));
    L.damp_f.push_back(take(k2 ? 4 * lbm::kDamp : 0));
    L.damp_ring.push_back(take(k2 ? 8 * 3 * lbm::kDamp : 0));
    L.proj.push_back(take(k2 ? 8 * lbm::kDamp * pctas : 0));
    L.drows.push_back(take(k2 && cfg->precision == 32 ? 4 * 6 * (size_t)c.ny : 0));
    L.pcount.push_back(take(k2 ? sizeof(unsigned) : 0));
    L.nu_ring.push_back(take(c.collision != 0 ? es * 3 * N : 0));
    L.Nmax = std::max(L.Nmax, N);
  }
  L.scratch_fields = lbm::kDiagFields;
  size_t pad = 0;  // the 12 prefix tables carry one extra row and column
  for (int m = 0; m < n; ++m)
    pad = std::max(pad, (size_t)cfg->members[m].nx + cfg->members[m].ny + 1);
  // slot 0 doubles as general staging (three snapshots, adjoint fields)
  L.slot_doubles = std::max(lbm::diag_slot_doubles(L.Nmax, pad),
                            ((size_t)L.scratch_fields * L.Nmax + 31) / 32 * 32);
  L.jpart_doubles = lbm::diag_job_partials(L.Nmax, pad);
  const size_t per_slot = 8 * (L.slot_doubles + L.jpart_doubles);
  size_t slots = cfg->diag_batch > 0 ? (size_t)cfg->diag_batch
                                     : std::max<size_t>(1, kDiagBatchBytes / per_slot);
  L.diag_slots = (int)std::min<size_t>(slots, (size_t)n);
  L.scratch = take(8 * L.slot_doubles * L.diag_slots);
  L.partials = take(8 * (size_t)lbm::kGeneralPartials);
  L.count = take(sizeof(unsigned));
  L.jpart = take(8 * L.jpart_doubles * L.diag_slots);
  L.jobs = take(sizeof(lbm::DiagJob) * n);
  L.stats = take(8 * (size_t)n * kMaxL * 30);
  L.edges = take(8 * 2 * (size_t)lbm::kDiagMaxEdges);
  L.hist = take(8 * (size_t)n * kMaxL * 3 * (lbm::kDiagMaxEdges + 1));
  L.mach = take(8 * (size_t)n * kMaxL * 2);
  L.Ls = take(4 * 8 * (size_t)n * kMaxL);  // per-size meta rows {L, boxes, offsets, out row}
  L.out7 = take(8 * 8);
  L.origin_cap = std::max<size_t>(4 * L.Nmax, (size_t)1 << 20);
  L.origins = take(8 * L.origin_cap);
  L.total = off;
  return L;
}

}  // namespace

struct lbm_handle {
  lbm_config cfg;
  std::vector<lbm_member_cfg> mcfg;
  std::vector<Member> hm;
  Layout lay;
  char *ws = nullptr;
  Member *d_members = nullptr;
  Tile *d_tiles = nullptr;
  int ntiles = 0;
  std::vector<int> scalar_members;
  int precision = 32;
  int diag_precision = 32;  // arithmetic of the term fields and box statistics
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t diag_stream = nullptr;  // asynchronous diagnostics
  cudaEvent_t ev_ready = nullptr, ev_diag_done = nullptr;
  bool diag_pending = false;
  bool has_kind2 = false;  // some member uses the paper's forcing (kind 2)
  bool proj_quad = true;   // every kind-2 member allows the four-cell projection
  bool has_vv = false;     // some member has a variable-viscosity collision
  bool has_elbm = false;   // some member has the entropic collision
  int cur = 0;
  long long t = 0;
  long long ring_time[3] = {-1, -1, -1};
  lbm::DiagScratch sc{};
  lbm::LaunchCfg lc{8, 1, 0, 0, 8};
  int graph_k = 0;
  cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};  // by storage state
  int persist_ctas = 0;  // > 0: one small general-kernel member, steps in one cooperative launch
  lbm::GridSync gsync{};
  float tuned_ms = 0.f;  // autotuned time of one step, ms (0: not tuned)
  long long launches = 0;  // kernels issued (graph replays count their nodes)
  std::string err = "no error";
};

namespace {

int fail(lbm_handle *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  g_last_error = msg;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(h, LBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

char *ws_at(lbm_handle *h, size_t off) { return h->ws + off; }

int build_tiles(lbm_handle *h) {
  std::vector<Tile> tiles;
  h->scalar_members.clear();
  const int rows = h->lc.block_warps_y * h->lc.rows_per_warp;
  for (int m = 0; m < (int)h->mcfg.size(); ++m) {
    const lbm_member_cfg &c = h->mcfg[m];
    if (!vector_eligible(c, h->precision)) {
      h->scalar_members.push_back(m);
      continue;
    }
    for (int y0 = 0; y0 < c.ny; y0 += rows)
      for (int x0 = 0; x0 < c.nx; x0 += kTileW) tiles.push_back(Tile{m, x0, y0, 0});
  }
  // With the paper forcing every step first projects the state member by
  // member in ascending order; the step then takes the members in descending
  // order, starting on those whose populations the projection read last
  // (still in L2), and leaves the lowest members freshly written for the
  // next projection.
  if (h->has_kind2) std::reverse(tiles.begin(), tiles.end());
  h->ntiles = (int)tiles.size();
  if (!tiles.empty())
    CK(cudaMemcpyAsync(h->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(),
                       cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

// Largest grid of the handle (batched per-member launches).
void max_grid(const lbm_handle *h, int *nx, int *ny) {
  *nx = 1;
  *ny = 1;
  for (const lbm_member_cfg &c : h->mcfg) {
    *nx = std::max(*nx, c.nx);
    *ny = std::max(*ny, c.ny);
  }
}

// Damping coefficients of eq. (16) of every kind-2 member for the state in
// storage `cur`: slot < 0 for the step about to run, else a ring slot.
int project(lbm_handle *h, cudaStream_t s, int cur, int slot) {
  int nx, ny;
  max_grid(h, &nx, &ny);
  CK(lbm::launch_projection(h->precision, h->d_members, (int)h->mcfg.size(), nx, ny, cur, slot,
                            h->proj_quad, h->lc.proj_rows, s));
  return LBM_OK;
}

// Steps alternate the direction in which they walk the tile table, so each
// one starts on the tiles the previous one wrote last (still in L2); with
// the paper forcing the projection walks the members in ascending order and
// the step always in descending order (the table is built reversed).
int tile_flip(const lbm_handle *h, int cur) { return h->has_kind2 ? 0 : (cur & 1); }

// One time step of every member on stream s (kind-2 members first get the
// damping of the state being collided).
int launch_one_step(lbm_handle *h, cudaStream_t s, int cur) {
  if (h->has_kind2)
    if (int rc = project(h, s, cur, -1)) return rc;
  if (h->ntiles > 0)
    CK(lbm::launch_step_f32_vec(h->d_members, h->d_tiles, h->ntiles, cur, tile_flip(h, cur), h->lc,
                                s));
  if (h->scalar_members.size() == 1) {
    const int m = h->scalar_members[0];
    CK(lbm::launch_step_scalar(h->precision, h->d_members, m, h->mcfg[m].nx, h->mcfg[m].ny, cur, s));
  } else if (!h->scalar_members.empty()) {
    int nx = 1, ny = 1;
    for (int m : h->scalar_members) {
      nx = std::max(nx, h->mcfg[m].nx);
      ny = std::max(ny, h->mcfg[m].ny);
    }
    CK(lbm::launch_step_scalar_batch(h->precision, h->d_members, h->scalar_members.data(),
                                     (int)h->scalar_members.size(), nx, ny, cur, s));
  }
  return LBM_OK;
}

long long kernels_per_step(const lbm_handle *h) {
  const long long ns = (long long)h->scalar_members.size();
  return (h->ntiles > 0 ? 1 : 0) + (ns + 255) / 256 + (h->has_kind2 ? 1 : 0);
}

void drop_graphs(lbm_handle *h) {
  for (auto &g : h->graph)
    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
}

int get_graph(lbm_handle *h, int cur, cudaGraphExec_t *out) {
  if (!h->graph[cur]) {
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int c = cur, rc = LBM_OK;
    for (int i = 0; i < h->graph_k && rc == LBM_OK; ++i) {
      rc = launch_one_step(h, h->cap_stream, c);
      c ^= 1;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc != LBM_OK) { if (g) cudaGraphDestroy(g); return rc; }
    CK(e);
    e = cudaGraphInstantiate(&h->graph[cur], g, 0);
    cudaGraphDestroy(g);
    CK(e);
  }
  *out = h->graph[cur];
  return LBM_OK;
}

int run_steps(lbm_handle *h, long long k) {
  if (h->persist_ctas > 0 && k >= 2) {  // a small grid: the whole run in one launch
    while (k > 0) {
      const int n = (int)std::min<long long>(k, 1 << 30);
      CK(lbm::launch_step_scalar_persistent(h->precision, h->d_members, h->scalar_members[0],
                                            h->cur, n, h->persist_ctas, h->gsync, h->stream));
      h->launches += 1;
      if (n & 1) h->cur ^= 1;
      h->t += n;
      k -= n;
    }
    return LBM_OK;
  }
  while (k > 0) {
    if (h->graph_k > 0 && k >= h->graph_k) {
      cudaGraphExec_t g;
      int rc = get_graph(h, h->cur, &g);
      if (rc) return rc;
      CK(cudaGraphLaunch(g, h->stream));
      h->launches += (long long)h->graph_k * kernels_per_step(h);
      k -= h->graph_k;
      h->t += h->graph_k;  // graph_k is even: buffer parity unchanged
    } else {
      int rc = launch_one_step(h, h->stream, h->cur);
      if (rc) return rc;
      h->launches += kernels_per_step(h);
      h->cur ^= 1;
      k -= 1;
      h->t += 1;
    }
  }
  return LBM_OK;
}

bool is_snap_time(const lbm_handle *h, long long t) {
  const long long D = h->cfg.diag_every;
  if (D <= 0) return false;
  const long long r = t % D;
  return r == 0 || r == D - 1 || r == D - 2;
}

double *snap_slot(lbm_handle *h, int m, int slot) {
  const size_t N = (size_t)h->mcfg[m].nx * h->mcfg[m].ny;
  return h->hm[m].snap + (size_t)slot * 3 * N;
}

// Orders the main stream after any asynchronous diagnostic still running:
// it reads the snapshot ring and uses the diagnostic scratch.
int wait_diag(lbm_handle *h) {
  if (h->diag_pending) CK(cudaStreamWaitEvent(h->stream, h->ev_diag_done, 0));
  return LBM_OK;
}

int record(lbm_handle *h) {
  if (int rc = wait_diag(h)) return rc;
  const int slot = (int)(h->t % 3);
  int nx = 1, ny = 1;
  for (const lbm_member_cfg &c : h->mcfg) {
    nx = std::max(nx, c.nx);
    ny = std::max(ny, c.ny);
  }
  // four cells per lane when every member is an FP32 vector-kernel member
  // with a constant viscosity (no local viscosity to record)
  const bool quad = h->precision == 32 && h->scalar_members.empty() && !h->has_vv;
  CK(lbm::launch_snapshot_ring(h->precision, h->d_members, (int)h->mcfg.size(), nx, ny, h->cur,
                               slot, quad, h->stream));
  h->launches += 1;
  if (h->has_kind2) {  // the damping of this state, for the diagnostic
    if (int rc = project(h, h->stream, h->cur, slot)) return rc;
    h->launches += 1;
  }
  h->ring_time[slot] = h->t;
  return LBM_OK;
}

int check_member(lbm_handle *h, int member) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (member < 0 || member >= (int)h->mcfg.size())
    return fail(h, LBM_ERR_ARG, "member index out of range");
  return LBM_OK;
}

// Autotune of the batched launch, run at create time while the populations
// are still undefined: each candidate (warps per CTA, rows per warp, grid
// size, and -- when the storage is left to the tuner -- double buffer
// versus in-place AA) is timed over 6 steps (both AA phases) on the live
// buffers, and the fastest is kept.  The state is reset to its initial
// phase afterwards.
int autotune(lbm_handle *h) {
  if (h->precision != 32) return LBM_OK;
  size_t cells = 0;
  for (auto &c : h->mcfg)
    if (vector_eligible(c, 32)) cells += (size_t)c.nx * c.ny;
  if (cells < (1u << 20)) return LBM_OK;  // small ensembles: default shape
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  struct Cand { lbm::LaunchCfg lc; int state; float ms; };
  std::vector<int> states;
  if (h->cfg.storage == 0) states = {0, 2};
  else states = {h->cfg.storage == 1 ? 2 : 0};
  std::vector<Cand> cands;
  for (int st : states)
    for (int wy : {4, 8})
      for (int rows : {1, 2, 4})
        for (int per : {0, 4, 8})
          cands.push_back({{wy, rows, per * nsm, h->lc.paper_force, h->lc.proj_rows}, st, 0.f});
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // 2 warm-up and `steps` timed steps of candidate i: ms per step
  auto time_candidate = [&](size_t i, int steps, float *ms) -> int {
    h->lc = cands[i].lc;
    int rc = build_tiles(h);
    if (rc) return rc;
    int st = cands[i].state;
    for (int w = 0; w < 2; ++w) {
      if ((rc = launch_one_step(h, h->stream, st))) return rc;
      st ^= 1;
    }
    CK(cudaEventRecord(e0, h->stream));
    for (int r = 0; r < steps; ++r) {
      if ((rc = launch_one_step(h, h->stream, st))) return rc;
      st ^= 1;
    }
    CK(cudaEventRecord(e1, h->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    *ms /= (float)steps;
    return LBM_OK;
  };
  int rc = LBM_OK;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess)
    rc = fail(h, LBM_ERR_CUDA, std::string("autotune events: ") + cudaGetErrorString(e));
  // every candidate once (6 steps), then the three fastest again, three runs
  // of 12 steps each: the median decides (single short runs are noisy)
  for (size_t i = 0; i < cands.size() && rc == LBM_OK; ++i)
    rc = time_candidate(i, 6, &cands[i].ms);
  std::vector<int> order(cands.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return cands[a].ms < cands[b].ms; });
  int best = order.empty() ? 0 : order[0];
  float best_ms = 1e30f;
  for (size_t k = 0; k < order.size() && k < 3 && rc == LBM_OK; ++k) {
    float t[3];
    for (int r = 0; r < 3 && rc == LBM_OK; ++r) rc = time_candidate(order[k], 12, &t[r]);
    if (rc != LBM_OK) break;
    std::sort(t, t + 3);
    if (t[1] < best_ms) {
      best_ms = t[1];
      best = order[k];
    }
  }
  // with the paper forcing, the rows per thread of the projection (its
  // pipelining depth and CTA count) on the chosen shape, timed likewise
  if (rc == LBM_OK && h->has_kind2 && h->proj_quad) {
    const Cand base = cands[best];
    for (int pr : {4, 16}) {
      if (rc != LBM_OK) break;
      if (pr == base.lc.proj_rows) continue;
      cands.push_back(base);
      cands.back().lc.proj_rows = pr;
      float t[3];
      for (int r = 0; r < 3 && rc == LBM_OK; ++r) rc = time_candidate(cands.size() - 1, 12, &t[r]);
      if (rc != LBM_OK) break;
      std::sort(t, t + 3);
      if (t[1] < best_ms) {
        best_ms = t[1];
        best = (int)cands.size() - 1;
      }
    }
  }
  // the events are released on every path
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc != LBM_OK) return rc;
  h->lc = cands[best].lc;
  h->cur = cands[best].state;
  h->tuned_ms = best_ms;
  return build_tiles(h);
}

}  // namespace

extern "C" {

int lbm_workspace_size(const lbm_config *cfg, size_t *bytes) {
  std::string err;
  int rc = check_config(cfg, err);
  if (rc) return fail(nullptr, rc, err);
  if (!bytes) return fail(nullptr, LBM_ERR_ARG, "bytes is NULL");
  *bytes = make_layout(cfg).total;
  return LBM_OK;
}

int lbm_create(const lbm_config *cfg, void *workspace, size_t bytes, lbm_handle **out) {
  std::string err;
  int rc = check_config(cfg, err);
  if (rc) return fail(nullptr, rc, err);
  if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  Layout lay = make_layout(cfg);
  if (!workspace || bytes < lay.total)
    return fail(nullptr, LBM_ERR_WORKSPACE, "workspace smaller than lbm_workspace_size()");
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign != 0)
    return fail(nullptr, LBM_ERR_WORKSPACE, "workspace must be 256-byte aligned");

  lbm_handle *h = new lbm_handle();
  h->cfg = *cfg;
  h->mcfg.assign(cfg->members, cfg->members + cfg->n_members);
  h->cfg.members = h->mcfg.data();
  h->lay = lay;
  h->ws = static_cast<char *>(workspace);
  h->precision = cfg->precision;
  h->diag_precision = cfg->diag_precision ? cfg->diag_precision : cfg->precision;
  h->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  h->graph_k = cfg->graph_steps > 0 ? (cfg->graph_steps + 1) / 2 * 2 : 0;
  h->d_members = reinterpret_cast<Member *>(ws_at(h, lay.members));
  h->d_tiles = reinterpret_cast<Tile *>(ws_at(h, lay.tiles));
  h->sc.f = reinterpret_cast<double *>(ws_at(h, lay.scratch));
  h->sc.N = lay.Nmax;
  h->sc.partials = reinterpret_cast<double *>(ws_at(h, lay.partials));
  h->sc.count = reinterpret_cast<unsigned *>(ws_at(h, lay.count));
  h->sc.slots = lay.diag_slots;
  h->sc.slot_doubles = lay.slot_doubles;
  h->sc.jpart = reinterpret_cast<double *>(ws_at(h, lay.jpart));
  h->sc.jpart_doubles = lay.jpart_doubles;

  auto cleanup = [&](int code) {
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->diag_stream) cudaStreamDestroy(h->diag_stream);
    if (h->ev_ready) cudaEventDestroy(h->ev_ready);
    if (h->ev_diag_done) cudaEventDestroy(h->ev_diag_done);
    delete h;
    return code;
  };
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->diag_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_ready, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_diag_done, cudaEventDisableTiming) != cudaSuccess)
    return cleanup(fail(nullptr, LBM_ERR_CUDA, "cannot create the streams and events"));

  const size_t es = h->precision == 32 ? 4 : 8;
  std::vector<char> tab;
  for (int m = 0; m < cfg->n_members; ++m) {
    const lbm_member_cfg &c = h->mcfg[m];
    Member M{};
    M.nx = c.nx;
    M.ny = c.ny;
    M.pitch = pitch_of(c.nx, h->precision);
    M.force_kind = c.force_kind;
    M.kf = c.kf;
    M.tau = c.tau;
    M.omega = 1.0 / c.tau;
    M.rho0 = c.rho0;
    M.F0 = c.F0;
    M.alpha = c.alpha;
    M.nu = (c.tau - 0.5) / 3.0;
    M.rho0_f = (float)c.rho0;
    M.omega_f = (float)(1.0 / c.tau);
    M.alpha_f = (float)c.alpha;
    M.plane = (size_t)c.ny * M.pitch;
    M.pop[0] = ws_at(h, lay.pop0[m]);
    M.pop[1] = ws_at(h, lay.pop1[m]);
    M.fx_tab = ws_at(h, lay.fx[m]);
    M.fy_tab = ws_at(h, lay.fy[m]);
    M.fx_tab64 = reinterpret_cast<double *>(ws_at(h, lay.fx64[m]));
    M.fy_tab64 = reinterpret_cast<double *>(ws_at(h, lay.fy64[m]));
    M.snap = reinterpret_cast<double *>(ws_at(h, lay.snap[m]));
    M.status = reinterpret_cast<int *>(ws_at(h, lay.status)) + m;
    M.collision = c.collision;
    M.Cs = c.Cs;
    M.Cs_f = (float)c.Cs;
    M.tau_f = (float)c.tau;
    if (c.collision != 0) {
      M.nu_ring = ws_at(h, lay.nu_ring[m]);
      h->has_vv = true;
      if (c.collision == 3) h->has_elbm = true;
    }
    if (c.force_kind == 2) {
      M.FR0 = c.FR0;
      M.ft_tab = ws_at(h, lay.ft[m]);
      M.ft_tab64 = reinterpret_cast<double *>(ws_at(h, lay.ft64[m]));
      M.trig = ws_at(h, lay.trig[m]);
      M.trig64 = reinterpret_cast<double *>(ws_at(h, lay.trig64[m]));
      M.damp = reinterpret_cast<double *>(ws_at(h, lay.damp[m]));
      M.damp_f = reinterpret_cast<float *>(ws_at(h, lay.damp_f[m]));
      M.damp_ring = reinterpret_cast<double *>(ws_at(h, lay.damp_ring[m]));
      M.proj_part = reinterpret_cast<double *>(ws_at(h, lay.proj[m]));
      M.damp_rows = h->precision == 32 ? reinterpret_cast<float *>(ws_at(h, lay.drows[m]))
                                       : nullptr;
      M.proj_count = reinterpret_cast<unsigned *>(ws_at(h, lay.pcount[m]));
      h->has_kind2 = true;
      if (h->precision != 32 || c.nx % 4 != 0) h->proj_quad = false;
    }
    h->hm.push_back(M);
    // Kolmogorov tables: F_ext,x(y) = F0 sin(2 pi kf y / ny), F_ext,y(x) likewise.
    std::vector<double> fx(c.ny, 0.0), fy(c.nx, 0.0);
    if (c.force_kind == 1) {
      const double pi = 3.14159265358979323846;
      for (int y = 0; y < c.ny; ++y) fx[y] = c.F0 * std::sin(2.0 * pi * c.kf * (double)y / c.ny);
      for (int x = 0; x < c.nx; ++x) fy[x] = c.F0 * std::sin(2.0 * pi * c.kf * (double)x / c.nx);
    }
    cudaStream_t s = h->stream;
    auto put = [&](void *dst, const std::vector<double> &v) -> cudaError_t {
      if (es == 8) return cudaMemcpyAsync(dst, v.data(), 8 * v.size(), cudaMemcpyHostToDevice, s);
      std::vector<float> f(v.begin(), v.end());
      cudaError_t e = cudaMemcpyAsync(dst, f.data(), 4 * f.size(), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // f is a temporary
      return e;
    };
    cudaError_t e = put(M.fx_tab, fx);
    if (e == cudaSuccess) e = put(M.fy_tab, fy);
    if (e == cudaSuccess) e = cudaMemcpyAsync(M.fx_tab64, fx.data(), 8 * fx.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(M.fy_tab64, fy.data(), 8 * fy.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(M.pop[0], 0, es * 9 * M.plane, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(M.pop[1], 0, es * 9 * M.plane, s);
    if (e == cudaSuccess && c.force_kind == 2) {
      std::vector<double> ft, ftp, trig;
      shell_force_tables(c, M.pitch, &ft, &ftp, &trig);
      e = put(M.ft_tab, ftp);
      if (e == cudaSuccess) e = put(M.trig, trig);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(M.ft_tab64, ft.data(), 8 * ft.size(), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(M.trig64, trig.data(), 8 * trig.size(), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(M.damp, 0, 8 * lbm::kDamp, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(M.damp_f, 0, 4 * lbm::kDamp, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(M.damp_ring, 0, 8 * 3 * lbm::kDamp, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(M.proj_count, 0, sizeof(unsigned), s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host tables are temporaries
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // fx/fy are temporaries
    if (e != cudaSuccess)
      return cleanup(fail(nullptr, LBM_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e)));
  }
  cudaError_t e = cudaMemcpyAsync(h->d_members, h->hm.data(), sizeof(Member) * h->hm.size(),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws_at(h, lay.status), 0, sizeof(int) * cfg->n_members, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->sc.count, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess)
    return cleanup(fail(nullptr, LBM_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e)));
  h->cur = cfg->storage == 1 ? 2 : 0;
  h->lc.paper_force = h->has_elbm ? 3 : (h->has_vv ? 2 : (h->has_kind2 ? 1 : 0));
  {
    unsigned *w = reinterpret_cast<unsigned *>(ws_at(h, lay.sync));
    h->gsync = lbm::GridSync{w, w + 1, reinterpret_cast<int *>(w + 2)};
    e = cudaMemsetAsync(w, 0, 4 * sizeof(unsigned), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess)
      return cleanup(fail(nullptr, LBM_ERR_CUDA, std::string("create: ") + cudaGetErrorString(e)));
  }
  rc = build_tiles(h);
  if (rc == LBM_OK) rc = autotune(h);
  if (rc != LBM_OK) {
    std::string msg = h->err;
    return cleanup(fail(nullptr, rc, msg));
  }
  // one small member on the general kernel without the paper forcing (whose
  // damping needs a projection launch per step), no graph replay asked for:
  // all the steps of a run in one cooperative launch
  {
    const lbm_member_cfg &c0 = h->mcfg[0];
    if (h->cfg.graph_steps == 0 && h->mcfg.size() == 1 && h->ntiles == 0 &&
        h->scalar_members.size() == 1 && !h->has_kind2 &&
        (long long)c0.nx * c0.ny < lbm::kPersistMaxCells)
      h->persist_ctas = lbm::persistent_ctas(h->precision, (long long)c0.nx * c0.ny);
  }
  *out = h;
  return LBM_OK;
}

int lbm_destroy(lbm_handle *h) {
  if (!h) return LBM_OK;
  if (h->diag_stream) cudaStreamSynchronize(h->diag_stream);
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->diag_stream) cudaStreamDestroy(h->diag_stream);
  if (h->ev_ready) cudaEventDestroy(h->ev_ready);
  if (h->ev_diag_done) cudaEventDestroy(h->ev_diag_done);
  delete h;
  return LBM_OK;
}

// The device's address of page-locked host memory (cudaHostAlloc /
// cudaHostRegister, e.g. a pinned torch tensor), or nullptr for pageable
// memory: init kernels read such fields in place over the host link.
const double *mapped_host(const double *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // pageable memory on older drivers: not an error here
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return static_cast<const double *>(a.devicePointer);
}

// Host fields all page-locked: their device addresses, read in place.
bool map_host_fields(const double *&r, const double *&u, const double *&v) {
  const double *mr = mapped_host(r), *mu = mapped_host(u), *mv = mapped_host(v);
  if (!mr || !mu || !mv) return false;
  r = mr;
  u = mu;
  v = mv;
  return true;
}

int lbm_init_fields(lbm_handle *h, int member, const double *rho, const double *ux,
                    const double *uy, int on_device) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (!rho || !ux || !uy) return fail(h, LBM_ERR_ARG, "rho/ux/uy must not be NULL");
  int m0 = member, m1 = member + 1;
  if (member < 0) { m0 = 0; m1 = (int)h->mcfg.size(); }
  else if (member >= (int)h->mcfg.size()) return fail(h, LBM_ERR_ARG, "member index out of range");
  const int nx = h->mcfg[m0].nx, ny = h->mcfg[m0].ny;
  for (int m = m0; m < m1; ++m)
    if (h->mcfg[m].nx != nx || h->mcfg[m].ny != ny)
      return fail(h, LBM_ERR_ARG, "shared init fields need equal grids");
  const size_t N = (size_t)nx * ny;
  const double *r = rho, *u = ux, *v = uy;
  if (!on_device && map_host_fields(r, u, v)) on_device = 1;  // page-locked: read in place
  // host fields are staged in the diagnostic scratch: wait for a queued
  // asynchronous diagnostic; device fields only overwrite the populations,
  // which the diagnostic never reads (it works on the snapshot ring)
  if (!on_device)
    if (int rc = wait_diag(h)) return rc;
  if (!on_device) {
    double *st = h->sc.f;  // staging: three scratch fields
    CK(cudaMemcpyAsync(st, rho, 8 * N, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(st + N, ux, 8 * N, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(st + 2 * N, uy, 8 * N, cudaMemcpyHostToDevice, h->stream));
    r = st; u = st + N; v = st + 2 * N;
  }
  if (h->cur >= 2) {
    // AA storage restarts at its even phase; members not re-initialised here
    // keep their data only when the phase already is even
    if (h->cur == 3 && m1 - m0 != (int)h->mcfg.size())
      return fail(h, LBM_ERR_ARG, "AA storage: initialise every member (or at an even step)");
    h->cur = 2;
  }
  for (int m = m0; m < m1; ++m)
    CK(lbm::launch_init_fields(h->precision, h->d_members, &m, 1, nx, ny, r, u, v, h->cur,
                               h->stream));
  h->launches += m1 - m0;
  if (!on_device) CK(cudaStreamSynchronize(h->stream));
  h->t = 0;
  h->ring_time[0] = h->ring_time[1] = h->ring_time[2] = -1;
  return LBM_OK;
}

int lbm_init_fields_batch(lbm_handle *h, const int *members, int n, const double *rho,
                          const double *ux, const double *uy, int on_device) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (!members || n < 1 || n > (int)h->mcfg.size())
    return fail(h, LBM_ERR_ARG, "need 1..n_members member indices");
  if (!rho || !ux || !uy) return fail(h, LBM_ERR_ARG, "rho/ux/uy must not be NULL");
  std::vector<char> seen(h->mcfg.size(), 0);
  for (int i = 0; i < n; ++i) {
    const int m = members[i];
    if (m < 0 || m >= (int)h->mcfg.size()) return fail(h, LBM_ERR_ARG, "member index out of range");
    if (seen[m]) return fail(h, LBM_ERR_ARG, "member listed twice");
    seen[m] = 1;
    if (h->mcfg[m].nx != h->mcfg[members[0]].nx || h->mcfg[m].ny != h->mcfg[members[0]].ny)
      return fail(h, LBM_ERR_ARG, "batched init fields need equal grids");
  }
  if (h->cur == 3 && n != (int)h->mcfg.size())
    return fail(h, LBM_ERR_ARG, "AA storage: initialise every member (or at an even step)");
  const int nx = h->mcfg[members[0]].nx, ny = h->mcfg[members[0]].ny;
  const size_t N = (size_t)nx * ny;
  if (!on_device && map_host_fields(rho, ux, uy)) on_device = 1;  // page-locked: read in place
  if (!on_device)  // staging in the diagnostic scratch (see lbm_init_fields)
    if (int rc = wait_diag(h)) return rc;
  if (h->cur >= 2) h->cur = 2;  // AA storage restarts at its even phase
  // host fields go through the diagnostic scratch (every slot) in chunks of
  // whole members: one copy per field and chunk, one synchronisation at the end
  const size_t cap = on_device ? (size_t)n : (size_t)h->sc.slots * h->sc.slot_doubles / (3 * N);
  if (cap < 1) return fail(h, LBM_ERR_WORKSPACE, "staging scratch smaller than one member");
  for (int i0 = 0; i0 < n; i0 += (int)std::min<size_t>(cap, (size_t)(n - i0))) {
    const int k = (int)std::min<size_t>(cap, (size_t)(n - i0));
    const double *r = rho + (size_t)i0 * N, *u = ux + (size_t)i0 * N, *v = uy + (size_t)i0 * N;
    if (!on_device) {
      double *st = h->sc.f;
      CK(cudaMemcpyAsync(st, r, 8 * N * k, cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(st + N * k, u, 8 * N * k, cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(st + 2 * N * k, v, 8 * N * k, cudaMemcpyHostToDevice, h->stream));
      r = st; u = st + N * k; v = st + 2 * N * k;
    }
    CK(lbm::launch_init_fields(h->precision, h->d_members, members + i0, k, nx, ny, r, u, v,
                               h->cur, h->stream));
    h->launches += (k + lbm::InitList::kMax - 1) / lbm::InitList::kMax;
  }
  if (!on_device) CK(cudaStreamSynchronize(h->stream));
  h->t = 0;
  h->ring_time[0] = h->ring_time[1] = h->ring_time[2] = -1;
  return LBM_OK;
}

long long lbm_time(const lbm_handle *h) { return h ? h->t : -1; }

long long lbm_launch_count(const lbm_handle *h) { return h ? h->launches : -1; }

long long lbm_kernels_per_step(const lbm_handle *h) { return h ? kernels_per_step(h) : -1; }

int lbm_set_launch(lbm_handle *h, int warps, int rows, int grid, int proj_rows) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (rows != 1 && rows != 2 && rows != 4) return fail(h, LBM_ERR_ARG, "rows must be 1, 2 or 4");
  if (grid < 0) return fail(h, LBM_ERR_ARG, "grid must be >= 0");
  if (warps < 1 || warps > 8) return fail(h, LBM_ERR_ARG, "warps must be 1..8");
  if (proj_rows < 0 || proj_rows > 64) return fail(h, LBM_ERR_ARG, "proj_rows must be 0..64");
  if (int rc = wait_diag(h)) return rc;
  drop_graphs(h);
  h->lc = lbm::LaunchCfg{warps, rows, grid, h->lc.paper_force,
                         proj_rows > 0 ? proj_rows : h->lc.proj_rows};
  h->tuned_ms = 0.f;
  return build_tiles(h);
}

int lbm_tuning(const lbm_handle *h, int *storage, int *warps, int *rows, int *grid,
               float *step_ms, int *proj_rows) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (proj_rows) *proj_rows = h->lc.proj_rows;
  if (storage) *storage = h->cur >= 2 ? 1 : 2;
  if (warps) *warps = h->lc.block_warps_y;
  if (rows) *rows = h->lc.rows_per_warp;
  if (grid) *grid = h->lc.grid_ctas;
  if (step_ms) *step_ms = h->tuned_ms;
  return LBM_OK;
}

// The snapshot of a state can be taken by the step that reads it (one
// launch instead of two) when every member runs in the FP32 vector kernel
// without the paper forcing or a variable viscosity.
bool fused_snapshots(const lbm_handle *h) {
  return h->precision == 32 && h->ntiles > 0 && h->scalar_members.empty() && !h->has_kind2 &&
         !h->has_vv && h->lc.paper_force == 0;
}

// One step of every member that also records the snapshot of the state it
// reads into the ring slot of the current time.
int step_recording(lbm_handle *h) {
  if (int rc = wait_diag(h)) return rc;
  const int slot = (int)(h->t % 3);
  CK(lbm::launch_step_f32_vec_snap(h->d_members, h->d_tiles, h->ntiles, h->cur,
                                   tile_flip(h, h->cur), h->lc, slot, h->stream));
  h->ring_time[slot] = h->t;
  h->launches += 1;
  h->cur ^= 1;
  h->t += 1;
  return LBM_OK;
}

int lbm_step(lbm_handle *h, int nsteps) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (nsteps < 0) return fail(h, LBM_ERR_ARG, "nsteps must be >= 0");
  const long long end = h->t + nsteps;
  while (h->t < end) {
    if (is_snap_time(h, h->t) && h->ring_time[h->t % 3] != h->t) {
      if (fused_snapshots(h)) {  // the step itself records it
        if (int rc = step_recording(h)) return rc;
        continue;
      }
      if (int rc = record(h)) return rc;
    }
    long long next = end;
    if (h->cfg.diag_every > 0) {
      long long s = h->t + 1;
      while (s < end && !is_snap_time(h, s)) {
        const long long D = h->cfg.diag_every;
        const long long r = s % D;
        s += (r < D - 2) ? (D - 2 - r) : 1;  // jump to the next candidate
      }
      next = std::min(end, s);
    }
    int rc = run_steps(h, next - h->t);
    if (rc) return rc;
  }
  if (is_snap_time(h, h->t) && h->ring_time[h->t % 3] != h->t) return record(h);
  return LBM_OK;
}

int lbm_record_snapshot(lbm_handle *h) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  return record(h);
}

int lbm_moments(lbm_handle *h, int member, double *rho, double *ux, double *uy,
                double *omega) {
  int rc = check_member(h, member);
  if (rc) return rc;
  if ((rc = wait_diag(h))) return rc;
  const lbm_member_cfg &c = h->mcfg[member];
  double *snap = h->sc.f;  // scratch fields 0..2
  if (c.force_kind == 2) {  // damping of the current state into Member::damp
    if ((rc = project(h, h->stream, h->cur, -1))) return rc;
    h->launches += 1;
  }
  CK(lbm::launch_snapshot(h->precision, h->d_members, member, c.nx, c.ny, h->cur, snap, h->stream));
  CK(lbm::diag_moments(h->hm[member], snap, rho, ux, uy, omega, h->sc, h->stream));
  h->launches += omega ? 3 : 2;
  return LBM_OK;
}

int lbm_global_balance(lbm_handle *h, int member, double *out) {
  int rc = check_member(h, member);
  if (rc) return rc;
  if (!out) return fail(h, LBM_ERR_ARG, "out is NULL");
  if ((rc = wait_diag(h))) return rc;
  const lbm_member_cfg &c = h->mcfg[member];
  double *snap = h->sc.f;
  double *out_dev = reinterpret_cast<double *>(ws_at(h, h->lay.out7));
  if (c.force_kind == 2) {  // damping of the current state into Member::damp
    if ((rc = project(h, h->stream, h->cur, -1))) return rc;
    h->launches += 1;
  }
  CK(lbm::launch_snapshot(h->precision, h->d_members, member, c.nx, c.ny, h->cur, snap, h->stream));
  CK(lbm::diag_global(h->hm[member], snap, h->sc, out_dev, h->stream));
  h->launches += 4;
  CK(cudaMemcpyAsync(out, out_dev, 8 * LBM_NGLOBAL, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

}  // extern "C"

namespace {

// Queues the diagnostic of each listed member (term fields, summed-area
// tables, box queries, statistics) and copies every member's statistics to
// the host with one synchronisation at the end.
// Host side of a distributions request (lbm_subvolume_distributions).
struct DistRequest {
  const double *delta_edges, *mach_edges;
  int n_delta, n_mach;
  long long *delta_hist, *mach_hist;  // [nm][nL][2][n_delta + 1], [nm][nL][n_mach + 1]
  double *mach_stats;                 // [nm][nL][2]
};

int check_edges(lbm_handle *h, const double *e, int n) {
  if (!e || n < 1 || n > lbm::kDiagMaxEdges)
    return fail(h, LBM_ERR_ARG, "need 1..256 bin edges");
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(e[i]) || (i > 0 && !(e[i] > e[i - 1])))
      return fail(h, LBM_ERR_ARG, "bin edges must be finite and strictly ascending");
  return LBM_OK;
}

int balance_members(lbm_handle *h, const int *members, int nm, const int *L, int nL,
                    const int *origins, const int *counts, double *stats_out,
                    double *per_box_out, double *stats_dev_out,
                    const DistRequest *dist = nullptr) {
  if (!L || nL < 1 || nL > kMaxL) return fail(h, LBM_ERR_ARG, "need 1..32 box sizes");
  if (!stats_out && !stats_dev_out && !dist) return fail(h, LBM_ERR_ARG, "stats output is NULL");
  if (dist) {
    if (int rc = check_edges(h, dist->delta_edges, dist->n_delta)) return rc;
    if (int rc = check_edges(h, dist->mach_edges, dist->n_mach)) return rc;
    if (!dist->delta_hist || !dist->mach_hist || !dist->mach_stats)
      return fail(h, LBM_ERR_ARG, "distribution outputs are NULL");
  }
  if (nm < 1) return fail(h, LBM_ERR_ARG, "no member given");
  if (per_box_out && nm != 1) return fail(h, LBM_ERR_ARG, "per_box_out needs one member");
  if ((origins == nullptr) != (counts == nullptr))
    return fail(h, LBM_ERR_ARG, "origins and counts go together (both NULL: all origins)");
  size_t total_boxes = 0;
  if (origins) {
    for (int i = 0; i < nL; ++i) {
      if (counts[i] < 1) return fail(h, LBM_ERR_ARG, "every box size needs at least one box");
      total_boxes += (size_t)counts[i];
    }
    if (total_boxes > h->lay.origin_cap)
      return fail(h, LBM_ERR_ARG, "too many boxes for the origin buffer");
  }
  int nx_min = 0, ny_min = 0;  // every origin must lie in every listed grid
  for (int i = 0; i < nm; ++i) {
    int rc = check_member(h, members[i]);
    if (rc) return rc;
    const lbm_member_cfg &c = h->mcfg[members[i]];
    nx_min = i ? std::min(nx_min, c.nx) : c.nx;
    ny_min = i ? std::min(ny_min, c.ny) : c.ny;
  }
  if (origins)
    for (size_t k = 0; k < total_boxes; ++k)
      if (origins[2 * k] < 0 || origins[2 * k] >= nx_min || origins[2 * k + 1] < 0 ||
          origins[2 * k + 1] >= ny_min)
        return fail(h, LBM_ERR_ARG, "origin outside the grid");
  // history n, n-1, n-2 (shared clock of all members)
  const long long t = h->t;
  if (h->ring_time[t % 3] != t) {
    int rc = record(h);
    if (rc) return rc;
  }
  if (t < 2 || h->ring_time[(t - 1) % 3] != t - 1 || h->ring_time[(t - 2) % 3] != t - 2)
    return fail(h, LBM_ERR_HISTORY, "snapshots of time n-1 and n-2 are missing");
  // per member: the sizes that fit its grid, with their box counts and offsets
  std::vector<std::vector<int>> where(nm);
  std::vector<int> meta((size_t)nm * kMaxL * 8, 0), maxb(nm, 0);
  for (int i = 0; i < nm; ++i) {
    const lbm_member_cfg &c = h->mcfg[members[i]];
    const int N = c.nx * c.ny;
    int ooff = 0, row = 0, k = 0;
    for (int q = 0; q < nL; ++q) {
      const int nb = origins ? counts[q] : N;
      if (L[q] >= 1 && L[q] <= c.nx && L[q] <= c.ny) {
        int *mrow = &meta[((size_t)i * kMaxL + k) * 8];
        mrow[0] = L[q];
        mrow[1] = nb;
        mrow[2] = origins ? ooff : -1;
        mrow[3] = row;
        mrow[4] = i * nL + q;  // row of the statistics output
        maxb[i] = std::max(maxb[i], nb);
        where[i].push_back(q);
        ++k;
      } else if (per_box_out) {
        return fail(h, LBM_ERR_ARG, "per_box_out needs every box size to fit the grid");
      }
      ooff += origins ? counts[q] : 0;
      row += nb;
    }
  }
  // asynchronous: on the diagnostic stream, after the work queued so far on
  // the main stream (the snapshots); synchronous: on the main stream, after
  // any asynchronous diagnostic still running (shared scratch).
  const bool async = stats_dev_out != nullptr;
  cudaStream_t s = h->stream;
  if (async) {
    CK(cudaEventRecord(h->ev_ready, h->stream));
    CK(cudaStreamWaitEvent(h->diag_stream, h->ev_ready, 0));
    s = h->diag_stream;
  } else if (h->diag_pending) {
    CK(cudaStreamWaitEvent(h->stream, h->ev_diag_done, 0));
  }
  int *meta_dev = reinterpret_cast<int *>(ws_at(h, h->lay.Ls));
  int *orig_dev = origins ? reinterpret_cast<int *>(ws_at(h, h->lay.origins)) : nullptr;
  double *stats_dev = async ? stats_dev_out : reinterpret_cast<double *>(ws_at(h, h->lay.stats));
  CK(cudaMemsetAsync(stats_dev, 0xff, 8 * (size_t)nm * nL * 30, s));  // all-ones bits: NaN
  lbm::DiagDist dd{};
  const size_t hrow = 3 * (size_t)(lbm::kDiagMaxEdges + 1);
  if (dist) {
    double *ed = reinterpret_cast<double *>(ws_at(h, h->lay.edges));
    CK(cudaMemcpyAsync(ed, dist->delta_edges, 8 * dist->n_delta, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ed + lbm::kDiagMaxEdges, dist->mach_edges, 8 * dist->n_mach,
                       cudaMemcpyHostToDevice, s));
    dd.delta_edges = ed;
    dd.mach_edges = ed + lbm::kDiagMaxEdges;
    dd.n_delta = dist->n_delta;
    dd.n_mach = dist->n_mach;
    dd.hist = reinterpret_cast<unsigned long long *>(ws_at(h, h->lay.hist));
    dd.mach = reinterpret_cast<double *>(ws_at(h, h->lay.mach));
    CK(cudaMemsetAsync(dd.hist, 0, 8 * (size_t)nm * nL * hrow, s));
    CK(cudaMemsetAsync(dd.mach, 0xff, 8 * (size_t)nm * nL * 2, s));
  }
  CK(cudaMemcpyAsync(meta_dev, meta.data(), 4 * meta.size(), cudaMemcpyHostToDevice, s));
  if (origins)
    CK(cudaMemcpyAsync(orig_dev, origins, 8 * total_boxes, cudaMemcpyHostToDevice, s));
  // one job per member with at least one fitting size; batches of up to
  // sc.slots jobs, each batch one set of ten launches
  std::vector<lbm::DiagJob> jobs;
  for (int i = 0; i < nm; ++i) {
    if (where[i].empty()) continue;
    const int m = members[i];
    const Member &hm = h->hm[m];
    const size_t slot = jobs.size() % (size_t)h->sc.slots;
    lbm::DiagJob J{};
    J.nx = hm.nx;
    J.ny = hm.ny;
    J.nu = hm.nu;
    J.alpha = hm.alpha;
    J.rho_ref = hm.rho0;
    J.fxt = hm.fx_tab64;
    J.fyt = hm.fy_tab64;
    J.fxt_f = h->precision == 32 ? static_cast<const float *>(hm.fx_tab) : nullptr;
    J.fyt_f = h->precision == 32 ? static_cast<const float *>(hm.fy_tab) : nullptr;
    J.nu_f = (float)hm.nu;
    J.alpha_f = (float)hm.alpha;
    J.rho_ref_f = (float)hm.rho0;
    J.s0 = snap_slot(h, m, (int)(t % 3));
    J.s1 = snap_slot(h, m, (int)((t - 1) % 3));
    J.s2 = snap_slot(h, m, (int)((t - 2) % 3));
    J.base = h->sc.f + slot * h->sc.slot_doubles;
    J.part = h->sc.jpart + slot * h->sc.jpart_doubles;
    J.meta = meta_dev + (size_t)i * kMaxL * 8;
    J.nL = (int)where[i].size();
    J.max_boxes = maxb[i];
    J.qblocks = lbm::diag_query_blocks(maxb[i], origins != nullptr,
                                       std::min(nm, h->sc.slots));
    J.force_kind = hm.force_kind;
    if (hm.collision != 0) {  // local viscosity recorded with the snapshot at n
      const size_t N = (size_t)hm.nx * hm.ny;
      if (h->precision == 32)
        J.nu_cell_f = static_cast<const float *>(hm.nu_ring) + (size_t)(t % 3) * N;
      else
        J.nu_cell_d = static_cast<const double *>(hm.nu_ring) + (size_t)(t % 3) * N;
    }
    if (hm.force_kind == 2) {  // damping coefficients recorded with each snapshot
      J.ft64 = hm.ft_tab64;
      J.trig64 = hm.trig64;
      for (int k = 0; k < 3; ++k)
        J.dc[k] = hm.damp_ring + (size_t)((t - k) % 3) * lbm::kDamp;
    }
    jobs.push_back(J);
  }
  if (!jobs.empty()) {
    auto *jobs_dev = reinterpret_cast<lbm::DiagJob *>(ws_at(h, h->lay.jobs));
    CK(cudaMemcpyAsync(jobs_dev, jobs.data(), sizeof(lbm::DiagJob) * jobs.size(),
                       cudaMemcpyHostToDevice, s));
    for (size_t j0 = 0; j0 < jobs.size(); j0 += (size_t)h->sc.slots) {
      const int G = (int)std::min(jobs.size() - j0, (size_t)h->sc.slots);
      CK(lbm::diag_balance(jobs.data() + j0, jobs_dev + j0, G, h->diag_precision,
                           h->precision == 32, orig_dev, stats_dev, per_box_out,
                           dist ? &dd : nullptr, s));
      h->launches += 10;  // 4 term passes, scales, strip sums, table builder, constants, query, statistics
    }
  }
  if (async) {
    CK(cudaEventRecord(h->ev_diag_done, h->diag_stream));
    h->diag_pending = true;
    return LBM_OK;
  }
  if (stats_out)
    CK(cudaMemcpyAsync(stats_out, stats_dev, 8 * (size_t)nm * nL * 30, cudaMemcpyDeviceToHost,
                       h->stream));
  std::vector<unsigned long long> hist;
  if (dist) {
    hist.resize((size_t)nm * nL * hrow);
    CK(cudaMemcpyAsync(hist.data(), dd.hist, 8 * hist.size(), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaMemcpyAsync(dist->mach_stats, dd.mach, 8 * (size_t)nm * nL * 2,
                       cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  if (dist) {  // rows [member][size][3][kDiagMaxEdges + 1] to the caller's layouts
    const int bd = dist->n_delta + 1, bm = dist->n_mach + 1;
    for (size_t r = 0; r < (size_t)nm * nL; ++r) {
      const unsigned long long *src = hist.data() + r * hrow;
      for (int q = 0; q < 2; ++q)
        for (int b = 0; b < bd; ++b)
          dist->delta_hist[(r * 2 + q) * bd + b] =
              (long long)src[(size_t)q * (lbm::kDiagMaxEdges + 1) + b];
      for (int b = 0; b < bm; ++b)
        dist->mach_hist[r * bm + b] = (long long)src[2 * (size_t)(lbm::kDiagMaxEdges + 1) + b];
    }
  }
  return LBM_OK;
}

}  // namespace

int lbm_subvolume_balance(lbm_handle *h, int member, const int *L, int nL, const int *origins,
                          const int *counts, double *stats_out, double *per_box_out) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (!stats_out) return fail(h, LBM_ERR_ARG, "stats_out is NULL");
  return balance_members(h, &member, 1, L, nL, origins, counts, stats_out, per_box_out,
                         nullptr);
}

int lbm_subvolume_balance_batch(lbm_handle *h, const int *members, int n_members, const int *L,
                                int nL, const int *origins, const int *counts,
                                double *stats_out) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (!members) return fail(h, LBM_ERR_ARG, "members is NULL");
  if (!stats_out) return fail(h, LBM_ERR_ARG, "stats_out is NULL");
  return balance_members(h, members, n_members, L, nL, origins, counts, stats_out, nullptr,
                         nullptr);
}

int lbm_subvolume_balance_async(lbm_handle *h, const int *members, int n_members, const int *L,
                                int nL, const int *origins, const int *counts,
                                double *stats_dev) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (!members) return fail(h, LBM_ERR_ARG, "members is NULL");
  if (!stats_dev) return fail(h, LBM_ERR_ARG, "stats_dev is NULL");
  return balance_members(h, members, n_members, L, nL, origins, counts, nullptr, nullptr,
                         stats_dev);
}

int lbm_subvolume_distributions(lbm_handle *h, const int *members, int n_members, const int *L,
                                int nL, const int *origins, const int *counts,
                                const double *delta_edges, int n_delta_edges,
                                const double *mach_edges, int n_mach_edges, double *stats_out,
                                long long *delta_hist_out, long long *mach_hist_out,
                                double *mach_stats_out) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (!members) return fail(h, LBM_ERR_ARG, "members is NULL");
  DistRequest d{delta_edges, mach_edges, n_delta_edges, n_mach_edges,
                delta_hist_out, mach_hist_out, mach_stats_out};
  return balance_members(h, members, n_members, L, nL, origins, counts, stats_out, nullptr,
                         nullptr, &d);
}

int lbm_diag_synchronize(lbm_handle *h) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (h->diag_pending) CK(cudaEventSynchronize(h->ev_diag_done));
  return LBM_OK;
}

extern "C" {

int lbm_get_populations(lbm_handle *h, int member, double *f, int on_device) {
  int rc = check_member(h, member);
  if (rc) return rc;
  if (!f) return fail(h, LBM_ERR_ARG, "f is NULL");
  const lbm_member_cfg &c = h->mcfg[member];
  const size_t N = (size_t)c.nx * c.ny;
  if ((rc = wait_diag(h))) return rc;
  double *dst = on_device ? f : h->sc.f;
  CK(lbm::launch_get_populations(h->precision, h->d_members, member, c.nx, c.ny, h->cur, dst, h->stream));
  h->launches += 1;
  if (!on_device) {
    CK(cudaMemcpyAsync(f, dst, 8 * 9 * N, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

int lbm_set_populations(lbm_handle *h, int member, const double *f, int on_device) {
  int rc = check_member(h, member);
  if (rc) return rc;
  if (!f) return fail(h, LBM_ERR_ARG, "f is NULL");
  const lbm_member_cfg &c = h->mcfg[member];
  const size_t N = (size_t)c.nx * c.ny;
  if ((rc = wait_diag(h))) return rc;
  const double *src = f;
  if (!on_device) {
    CK(cudaMemcpyAsync(h->sc.f, f, 8 * 9 * N, cudaMemcpyHostToDevice, h->stream));
    src = h->sc.f;
  }
  CK(lbm::launch_set_populations(h->precision, h->d_members, member, c.nx, c.ny, h->cur, src, h->stream));
  h->launches += 1;
  if (!on_device) CK(cudaStreamSynchronize(h->stream));
  h->ring_time[0] = h->ring_time[1] = h->ring_time[2] = -1;
  return LBM_OK;
}

int lbm_member_status(lbm_handle *h, int member, int *status) {
  int rc = check_member(h, member);
  if (rc) return rc;
  if (!status) return fail(h, LBM_ERR_ARG, "status is NULL");
  const lbm_member_cfg &c = h->mcfg[member];
  CK(cudaMemsetAsync(h->hm[member].status, 0, sizeof(int), h->stream));
  CK(lbm::launch_status(h->precision, h->d_members, member, c.nx, c.ny, h->cur, h->stream));
  h->launches += 1;
  CK(cudaMemcpyAsync(status, h->hm[member].status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  int gave_up = 0;
  CK(cudaMemcpyAsync(&gave_up, h->gsync.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (gave_up)
    return fail(h, LBM_ERR_TIMEOUT,
                "a persistent step kernel gave up waiting for another CTA (grid barrier or "
                "damping coefficients)");
  return LBM_OK;
}

int lbm_adjoint_step(lbm_handle *h, int member, const double *f_n, const double *lambda_in,
                     double *lambda_out, double obj_weight, int bx, int by, int L,
                     double *dJ_dtau, double *dJ_dF0) {
  int rc = check_member(h, member);
  if (rc) return rc;
  const lbm_member_cfg &c = h->mcfg[member];
  if (c.force_kind == 2)
    return fail(h, LBM_ERR_ARG, "the adjoint supports force kinds 0 and 1 (the damping of "
                                "kind 2 couples every cell)");
  if (c.collision != 0)
    return fail(h, LBM_ERR_ARG, "the adjoint supports the BGK collision only");
  if (!f_n || !lambda_out) return fail(h, LBM_ERR_ARG, "f_n and lambda_out must not be NULL");
  if (lambda_in == lambda_out) return fail(h, LBM_ERR_ARG, "lambda_out may not alias lambda_in");
  if (!std::isfinite(obj_weight)) return fail(h, LBM_ERR_ARG, "obj_weight not finite");
  if (obj_weight != 0.0 &&
      (L < 1 || L > c.nx || L > c.ny || bx < 0 || bx >= c.nx || by < 0 || by >= c.ny))
    return fail(h, LBM_ERR_ARG, "objective box outside the grid");
  if ((rc = wait_diag(h))) return rc;
  CK(lbm::adjoint_step(h->hm[member], f_n, lambda_in, lambda_out, obj_weight, bx, by, L,
                       dJ_dtau, dJ_dF0, h->sc, h->stream));
  h->launches += lbm::adjoint_kernel_count(obj_weight);
  return LBM_OK;
}

int lbm_objective_accumulate(lbm_handle *h, int member, double weight, int bx, int by, int L,
                             double *acc) {
  int rc = check_member(h, member);
  if (rc) return rc;
  const lbm_member_cfg &c = h->mcfg[member];
  if (c.force_kind == 2 || c.collision != 0)
    return fail(h, LBM_ERR_ARG, "the objective supports force kinds 0 and 1 with BGK");
  if (!acc) return fail(h, LBM_ERR_ARG, "acc is NULL");
  if (L < 1 || L > c.nx || L > c.ny || bx < 0 || bx >= c.nx || by < 0 || by >= c.ny)
    return fail(h, LBM_ERR_ARG, "objective box outside the grid");
  if ((rc = wait_diag(h))) return rc;
  CK(lbm::objective_tiles(h->precision, h->d_members, member, h->hm[member], h->cur, weight, bx,
                          by, L, acc, h->sc, h->stream));
  h->launches += 1;
  return LBM_OK;
}

int lbm_objective_steps(lbm_handle *h, int member, int nsteps, double weight, int bx, int by,
                        int L, double *acc) {
  if (!h) return fail(nullptr, LBM_ERR_ARG, "handle is NULL");
  if (nsteps < 0) return fail(h, LBM_ERR_ARG, "nsteps must be >= 0");
  for (int k = 0; k < nsteps; ++k) {
    if (int rc = lbm_objective_accumulate(h, member, weight, bx, by, L, acc)) return rc;
    if (int rc = lbm_step(h, 1)) return rc;
  }
  return LBM_OK;
}

int lbm_record_trajectory(lbm_handle *h, int member, int nstates, double *states) {
  int rc = check_member(h, member);
  if (rc) return rc;
  if (!states) return fail(h, LBM_ERR_ARG, "states is NULL");
  if (nstates < 1) return fail(h, LBM_ERR_ARG, "nstates must be >= 1");
  const lbm_member_cfg &c = h->mcfg[member];
  const size_t N = (size_t)c.nx * c.ny;
  // one member on the general kernel, no snapshot cadence, no projection:
  // each step writes the public state it starts from (one launch and one
  // read of the state per level instead of a step and an export)
  if (h->mcfg.size() == 1 && h->scalar_members.size() == 1 && h->ntiles == 0 &&
      h->cfg.diag_every == 0 && !h->has_kind2) {
    if ((rc = wait_diag(h))) return rc;
    for (int k = 0; k + 1 < nstates; ++k) {
      CK(lbm::launch_step_scalar(h->precision, h->d_members, member, c.nx, c.ny, h->cur,
                                 h->stream, states + (size_t)k * 9 * N));
      h->launches += 1;
      h->cur ^= 1;
      h->t += 1;
    }
    return lbm_get_populations(h, member, states + (size_t)(nstates - 1) * 9 * N, 1);
  }
  for (int k = 0; k < nstates; ++k) {
    if (k > 0)
      if ((rc = lbm_step(h, 1))) return rc;
    if ((rc = lbm_get_populations(h, member, states + (size_t)k * 9 * N, 1))) return rc;
  }
  return LBM_OK;
}

int lbm_adjoint_sweep(lbm_handle *h, int member, const double *states, int nstates,
                      const double *lambda_in, double *lambda_out, double *lambda_tmp,
                      const double *weights, int bx, int by, int L, double *dJ_dtau,
                      double *dJ_dF0) {
  int rc = check_member(h, member);
  if (rc) return rc;
  if (!states || !lambda_out || !lambda_tmp || !weights)
    return fail(h, LBM_ERR_ARG, "states, lambda_out, lambda_tmp and weights must not be NULL");
  if (nstates < 1) return fail(h, LBM_ERR_ARG, "nstates must be >= 1");
  if (lambda_out == lambda_tmp || lambda_in == lambda_out || lambda_in == lambda_tmp)
    return fail(h, LBM_ERR_ARG, "lambda_in, lambda_out and lambda_tmp must be distinct");
  const lbm_member_cfg &c = h->mcfg[member];
  if (c.force_kind == 2)
    return fail(h, LBM_ERR_ARG, "the adjoint supports force kinds 0 and 1 (the damping of "
                                "kind 2 couples every cell)");
  if (c.collision != 0)
    return fail(h, LBM_ERR_ARG, "the adjoint supports the BGK collision only");
  bool any_obj = false;
  for (int k = 0; k < nstates; ++k) {
    if (!std::isfinite(weights[k])) return fail(h, LBM_ERR_ARG, "weights must be finite");
    any_obj = any_obj || weights[k] != 0.0;
  }
  if (any_obj && (L < 1 || L > c.nx || L > c.ny || bx < 0 || bx >= c.nx || by < 0 || by >= c.ny))
    return fail(h, LBM_ERR_ARG, "objective box outside the grid");
  if ((rc = wait_diag(h))) return rc;
  CK(lbm::adjoint_sweep(h->hm[member], states, nstates, lambda_in, lambda_out, lambda_tmp,
                        weights, bx, by, L, dJ_dtau, dJ_dF0, h->sc, h->stream, &h->launches));
  return LBM_OK;
}

int lbm_probe_fma_rate(int bits, void *cuda_stream, double *flops_per_s) {
  if (bits != 32 && bits != 64) return fail(nullptr, LBM_ERR_ARG, "bits must be 32 or 64");
  if (!flops_per_s) return fail(nullptr, LBM_ERR_ARG, "flops_per_s is NULL");
  cudaError_t e = lbm::probe_fma_rate(bits, static_cast<cudaStream_t>(cuda_stream), flops_per_s);
  if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_probe_grid_barrier(int ctas, int rounds, int withhold, void *cuda_stream,
                           int *gave_up) {
  if (ctas < 1 || ctas > 4096 || rounds < 0 || withhold >= ctas || !gave_up)
    return fail(nullptr, LBM_ERR_ARG, "need 1 <= ctas <= 4096, rounds >= 0, withhold < ctas");
  cudaError_t e = lbm::barrier_probe(ctas, rounds, withhold,
                                     static_cast<cudaStream_t>(cuda_stream), gave_up);
  if (e != cudaSuccess) return fail(nullptr, LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

const char *lbm_last_error(const lbm_handle *h) {
  return h ? h->err.c_str() : g_last_error.c_str();
}

}  // extern "C"

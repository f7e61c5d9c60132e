// C ABI of libsnap: argument checking, problem construction (row list, Jacobian pattern,
// implied rows), workspace sizing and dispatch to the kernels.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "kern_1dflux.h"
#include "snap_internal.h"

namespace {

thread_local char g_err[512] = "";
thread_local int g_launches = 0;

snap_status fail(snap_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

snap_status cuda_fail(cudaError_t e, const char *what) {
  return fail(SNAP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

SolverOpts to_solver(const snap_options &o) {
  SolverOpts s;
  s.tol_kkt = o.tol_kkt;
  s.tol_h = o.tol_h;
  s.c1 = o.armijo_c1;
  s.delta0 = o.delta0;
  s.w_keep = o.w_keep;
  s.max_iter = o.max_iter;
  s.max_backtracks = o.max_backtracks;
  s.max_corrections = o.max_corrections;
  s.pad = 0;
  return s;
}

snap_status check_opts(const snap_options &o) {
  if (!(o.tol_kkt > 0.0) || !(o.tol_h > 0.0) || o.max_iter < 0 || o.max_iter > 10000 ||
      o.max_backtracks < 0 || o.max_backtracks > 200 ||
      !(o.armijo_c1 > 0.0 && o.armijo_c1 < 0.5) || !(o.delta0 > 0.0) || o.max_corrections < 0 ||
      o.max_corrections > 100 ||
      o.path < SNAP_PATH_AUTO || o.path > SNAP_PATH_MIXED || !(o.w_keep >= 0.0 && o.w_keep < 1.0))
    return fail(SNAP_ERR_INVALID_ARG, "invalid snap_options");
  return SNAP_OK;
}

// Row list and CSR pattern of the 1-D families (nominal rows, columns ascending).
void build_pattern_1d(snap_problem *p) {
  const Geom1D &g = p->g1;
  std::vector<int> rp(1, 0), ci;
  std::vector<unsigned char> act;
  for (int i = 0; i < g.nx; ++i) { ci.push_back(i); rp.push_back((int)ci.size()); act.push_back(1); }
  if (g.rows & SL_MASS)
    for (int k = 0; k < g.nt; ++k) {
      for (int i = 0; i < g.nx; ++i) ci.push_back(k * g.nx + i);
      rp.push_back((int)ci.size()); act.push_back(k > 0);
    }
  if (g.rows & SL_ENERGY)
    for (int k = 0; k < g.nt; ++k) {
      for (int i = 0; i < g.nx; ++i) ci.push_back(k * g.nx + i);
      rp.push_back((int)ci.size()); act.push_back(k > 0);
    }
  if (g.rows & SL_BOUND)
    for (int k = 0; k < g.nt; ++k) {
      ci.push_back(k * g.nx); ci.push_back(k * g.nx + g.ih);
      rp.push_back((int)ci.size()); act.push_back(k > 0);
    }
  p->row_ptr = (int *)malloc(sizeof(int) * rp.size());
  p->col_idx = (int *)malloc(sizeof(int) * (ci.size() + 1));
  p->active = (unsigned char *)malloc(act.size() + 1);
  memcpy(p->row_ptr, rp.data(), sizeof(int) * rp.size());
  memcpy(p->col_idx, ci.data(), sizeof(int) * ci.size());
  memcpy(p->active, act.data(), act.size());
  p->info.pattern_nnz = (long long)ci.size();
  int na = 0;
  for (unsigned char a : act) na += a;
  p->info.n_rows_active = na;
}

// Appendix C toy family: IC rows, then left-Riemann mass differences for k = 2..nt.
void build_pattern_toy(snap_problem *p, int nx, int nt) {
  std::vector<int> rp(1, 0), ci;
  for (int i = 0; i < nx; ++i) { ci.push_back(i); rp.push_back((int)ci.size()); }
  for (int k = 1; k < nt; ++k) {
    for (int i = 0; i < nx - 1; ++i) ci.push_back(i);
    for (int i = 0; i < nx - 1; ++i) ci.push_back(k * nx + i);
    rp.push_back((int)ci.size());
  }
  const int m = (int)rp.size() - 1;
  p->row_ptr = (int *)malloc(sizeof(int) * rp.size());
  p->col_idx = (int *)malloc(sizeof(int) * (ci.size() + 1));
  p->active = (unsigned char *)malloc(m + 1);
  memcpy(p->row_ptr, rp.data(), sizeof(int) * rp.size());
  memcpy(p->col_idx, ci.data(), sizeof(int) * ci.size());
  memset(p->active, 1, m);
  p->info.pattern_nnz = (long long)ci.size();
  p->info.n_rows_active = m;
  p->info.n_rows_nominal = m;
}

// Family D: per slice a Dirichlet row (x_0), then the mass rows, then the Neumann rows
// (x_{nx-2}, x_{nx-1}); grouped by type: D rows 0..nt-1, M rows nt..2nt-1, N rows 2nt..3nt-1.
void build_pattern_bc(snap_problem *p, int nx, int nt) {
  std::vector<int> rp(1, 0), ci;
  for (int k = 0; k < nt; ++k) { ci.push_back(k * nx); rp.push_back((int)ci.size()); }
  for (int k = 0; k < nt; ++k) {
    for (int i = 0; i < nx; ++i) ci.push_back(k * nx + i);
    rp.push_back((int)ci.size());
  }
  for (int k = 0; k < nt; ++k) {
    ci.push_back(k * nx + nx - 2); ci.push_back(k * nx + nx - 1);
    rp.push_back((int)ci.size());
  }
  const int m = (int)rp.size() - 1;
  p->row_ptr = (int *)malloc(sizeof(int) * rp.size());
  p->col_idx = (int *)malloc(sizeof(int) * (ci.size() + 1));
  p->active = (unsigned char *)malloc(m + 1);
  memcpy(p->row_ptr, rp.data(), sizeof(int) * rp.size());
  memcpy(p->col_idx, ci.data(), sizeof(int) * ci.size());
  memset(p->active, 1, m);
  p->info.pattern_nnz = (long long)ci.size();
  p->info.n_rows_active = m;
}

// 1-D family E: IC rows, mass rows (those of slices 0..K implied: inactive), then the flux
// rows of steps 1..K (u^k_i and u^{k-1}_{i-1,i,i+1}, periodic).
void build_pattern_flux(snap_problem *p, int nx, int nt, int K) {
  std::vector<int> rp(1, 0), ci;
  std::vector<unsigned char> act;
  for (int i = 0; i < nx; ++i) { ci.push_back(i); rp.push_back((int)ci.size()); act.push_back(1); }
  for (int k = 0; k < nt; ++k) {
    for (int i = 0; i < nx; ++i) ci.push_back(k * nx + i);
    rp.push_back((int)ci.size());
    act.push_back(k > K ? 1 : 0);
  }
  for (int k = 1; k <= K; ++k)
    for (int i = 0; i < nx; ++i) {
      const int prev = (k - 1) * nx;
      ci.push_back(prev + (i + nx - 1) % nx);
      ci.push_back(prev + i);
      ci.push_back(prev + (i + 1) % nx);
      ci.push_back(k * nx + i);
      rp.push_back((int)ci.size());
      act.push_back(1);
    }
  const int m = (int)rp.size() - 1;
  p->row_ptr = (int *)malloc(sizeof(int) * rp.size());
  p->col_idx = (int *)malloc(sizeof(int) * (ci.size() + 1));
  p->active = (unsigned char *)malloc(m + 1);
  memcpy(p->row_ptr, rp.data(), sizeof(int) * rp.size());
  memcpy(p->col_idx, ci.data(), sizeof(int) * ci.size());
  memcpy(p->active, act.data(), m);
  int na = 0;
  for (unsigned char a : act) na += a;
  p->info.pattern_nnz = (long long)ci.size();
  p->info.n_rows_active = na;
}

// Family F (heat): IC rows, mass rows (implied), Crank-Nicolson rows k = 1..nt-1 (three
// stencil columns in slices k-1 and k), energy rows (implied; every column of slices k-1, k).
void build_pattern_heat(snap_problem *p, int nx, int nt) {
  std::vector<int> rp(1, 0), ci;
  std::vector<unsigned char> act;
  for (int i = 0; i < nx; ++i) { ci.push_back(i); rp.push_back((int)ci.size()); act.push_back(1); }
  for (int k = 0; k < nt; ++k) {
    for (int i = 0; i < nx; ++i) ci.push_back(k * nx + i);
    rp.push_back((int)ci.size());
    act.push_back(0);
  }
  for (int k = 1; k < nt; ++k)
    for (int i = 0; i < nx; ++i) {
      std::vector<int> c;
      for (int kk = k - 1; kk <= k; ++kk)
        for (int d = -1; d <= 1; ++d) c.push_back(kk * nx + (i + d + nx) % nx);
      std::sort(c.begin(), c.end());
      c.erase(std::unique(c.begin(), c.end()), c.end());
      ci.insert(ci.end(), c.begin(), c.end());
      rp.push_back((int)ci.size());
      act.push_back(1);
    }
  for (int k = 1; k < nt; ++k) {
    for (int i = 0; i < 2 * nx; ++i) ci.push_back((k - 1) * nx + i);
    rp.push_back((int)ci.size());
    act.push_back(0);
  }
  const int m = (int)rp.size() - 1;
  p->row_ptr = (int *)malloc(sizeof(int) * rp.size());
  p->col_idx = (int *)malloc(sizeof(int) * (ci.size() + 1));
  p->active = (unsigned char *)malloc(m + 1);
  memcpy(p->row_ptr, rp.data(), sizeof(int) * rp.size());
  memcpy(p->col_idx, ci.data(), sizeof(int) * ci.size());
  memcpy(p->active, act.data(), m);
  int na = 0;
  for (unsigned char a : act) na += a;
  p->info.pattern_nnz = (long long)ci.size();
  p->info.n_rows_active = na;
}

// 2-D family C: divergence rows [f][j][i] (4 stencil columns), then one energy row per frame.
void build_pattern_2d(snap_problem *p, int N, int nt) {
  std::vector<int> rp(1, 0), ci;
  std::vector<unsigned char> act;
  const int nf = 2 * N * N;
  for (int f = 0; f < nt; ++f)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        int c[4] = {f * nf + j * N + (i + N - 1) % N, f * nf + j * N + (i + 1) % N,
                    f * nf + N * N + ((j + N - 1) % N) * N + i, f * nf + N * N + ((j + 1) % N) * N + i};
        // ascending order within the row
        for (int a = 0; a < 4; ++a)
          for (int b2 = a + 1; b2 < 4; ++b2)
            if (c[b2] < c[a]) { int t = c[a]; c[a] = c[b2]; c[b2] = t; }
        for (int a = 0; a < 4; ++a) ci.push_back(c[a]);
        rp.push_back((int)ci.size());
        act.push_back(!((i < 2) && (j < 2)));
      }
  for (int f = 0; f < nt; ++f) {
    for (int v = 0; v < nf; ++v) ci.push_back(f * nf + v);
    rp.push_back((int)ci.size());
    act.push_back(1);
  }
  p->row_ptr = (int *)malloc(sizeof(int) * rp.size());
  p->col_idx = (int *)malloc(sizeof(int) * (ci.size() + 1));
  p->active = (unsigned char *)malloc(act.size() + 1);
  memcpy(p->row_ptr, rp.data(), sizeof(int) * rp.size());
  memcpy(p->col_idx, ci.data(), sizeof(int) * ci.size());
  memcpy(p->active, act.data(), act.size());
  p->info.pattern_nnz = (long long)ci.size();
  int na = 0;
  for (unsigned char a : act) na += a;
  p->info.n_rows_active = na;
}

snap_status check_batch(const snap_problem *p, int B) {
  if (!p) return fail(SNAP_ERR_INVALID_ARG, "null problem");
  if (B < 0) return fail(SNAP_ERR_INVALID_ARG, "negative batch size %d", B);
  if (p->desc.max_batch > 0 && B > p->desc.max_batch)
    return fail(SNAP_ERR_INVALID_ARG, "batch size %d exceeds max_batch %d", B, p->desc.max_batch);
  if ((long long)B * p->info.n_vars > (1LL << 40))
    return fail(SNAP_ERR_INVALID_ARG, "batch too large");
  return SNAP_OK;
}

size_t ws_bytes(const snap_problem *p, int B) {
  if (p->desc.family == SNAP_FAMILY_F_HEAT_ENERGY) return 0;
  if (p->desc.family == SNAP_FAMILY_C_DIV_ENERGY) return ws_bytes_2d(p, B);
  if (p->desc.family == SNAP_FAMILY_D_BURGERS_BC) return ws_bytes_1dbc(p, B);
  if (p->desc.family == SNAP_FAMILY_E_BURGERS_FLUX) return ws_bytes_1dflux(p, B);
  return ws_bytes_1d(p, B);
}

}  // namespace

void snap_note_launch(int n) { g_launches += n; }

void snap_reset_launches() { g_launches = 0; }

void snap_clear_error() { g_err[0] = 0; }

snap_status snap_fail_msg(snap_status st, const char *msg) { return fail(st, "%s", msg); }

snap_status snap_check_options(const snap_options &o) { return check_opts(o); }

extern "C" {

const char *snap_last_error(void) { return g_err; }

#ifdef SNAP_BOUNDS_CHECK
}  // extern "C"
__device__ unsigned long long g_snap_bounds_err = 0ull;
extern "C" {
snap_status snap_bounds_error(unsigned long long *word, int clear) {
  if (!word) return fail(SNAP_ERR_INVALID_ARG, "null output");
  cudaError_t e = cudaMemcpyFromSymbol(word, g_snap_bounds_err, sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "reading the bounds error word");
  if (clear) {
    const unsigned long long zero = 0ull;
    e = cudaMemcpyToSymbol(g_snap_bounds_err, &zero, sizeof(zero));
    if (e != cudaSuccess) return cuda_fail(e, "clearing the bounds error word");
  }
  return SNAP_OK;
}
#else
snap_status snap_bounds_error(unsigned long long *word, int clear) {
  (void)clear;
  if (word) *word = 0ull;
  return fail(SNAP_ERR_UNSUPPORTED, "this library was built without SNAP_BOUNDS_CHECK");
}
#endif

const char *snap_version(void) { return SNAP_VERSION_STRING; }

int snap_last_launch_count(void) { return g_launches; }

snap_status snap_options_default(snap_options *opt) {
  if (!opt) return fail(SNAP_ERR_INVALID_ARG, "null options");
  opt->tol_kkt = 1e-10;
  opt->tol_h = 1e-8;
  opt->max_iter = 50;
  opt->max_backtracks = 30;
  opt->armijo_c1 = 1e-4;
  opt->delta0 = 1e-8;
  opt->max_corrections = 0;
  opt->path = SNAP_PATH_AUTO;
  opt->w_keep = 0.01;
  return SNAP_OK;
}

snap_status snap_problem_create(const snap_problem_desc *d, snap_problem_t *out) {
  g_err[0] = 0;
  if (!d || !out) return fail(SNAP_ERR_INVALID_ARG, "null descriptor or output");
  if (d->nt < 2 || d->nt > (1 << 20)) return fail(SNAP_ERR_INVALID_ARG, "nt must be in [2, 2^20]");
  if (d->max_batch < 0) return fail(SNAP_ERR_INVALID_ARG, "max_batch must be >= 0");
  if (d->family != SNAP_FAMILY_E_BURGERS_FLUX && d->n_flux != 0)
    return fail(SNAP_ERR_INVALID_ARG, "n_flux is a family E field (must be 0)");
  snap_problem *p = (snap_problem *)calloc(1, sizeof(snap_problem));
  if (!p) return fail(SNAP_ERR_NO_MEMORY, "host allocation failed");
  p->desc = *d;
  switch (d->family) {
    case SNAP_FAMILY_A_MASS_ENERGY:
    case SNAP_FAMILY_B_BURGERS_BOUNDARY: {
      if (d->nx < 4 || (d->nx & 1) || d->nx > 512) {
        free(p);
        return fail(SNAP_ERR_INVALID_ARG, "1-D nx must be even and in [4, 512] (got %d)", d->nx);
      }
      unsigned rows = d->rows;
      if (rows == 0)
        rows = SNAP_ROW_IC | SNAP_ROW_MASS | SNAP_ROW_ENERGY |
               (d->family == SNAP_FAMILY_B_BURGERS_BOUNDARY ? SNAP_ROW_BOUNDARY : 0);
      if (!(rows & SNAP_ROW_IC) || (rows & ~15u) ||
          ((rows & SNAP_ROW_BOUNDARY) && d->family != SNAP_FAMILY_B_BURGERS_BOUNDARY)) {
        free(p);
        return fail(SNAP_ERR_INVALID_ARG, "invalid row mask 0x%x for family %d", rows, d->family);
      }
      if (!(d->energy_floor == d->energy_floor)) {
        free(p);
        return fail(SNAP_ERR_INVALID_ARG, "energy_floor is NaN");
      }
      Geom1D &g = p->g1;
      g.nx = d->nx;
      g.nt = d->nt;
      g.ih = d->nx / 2;
      g.rows = ((rows & SNAP_ROW_MASS) ? SL_MASS : 0) | ((rows & SNAP_ROW_ENERGY) ? SL_ENERGY : 0) |
               ((rows & SNAP_ROW_BOUNDARY) ? SL_BOUND : 0);
      g.has_ic = 1;
      g.dx = 1.0 / d->nx;
      g.energy_floor = d->energy_floor;
      g.n_vars = d->nx * d->nt;
      int off = d->nx;
      g.off_mass = (g.rows & SL_MASS) ? off : -1;
      off += (g.rows & SL_MASS) ? d->nt : 0;
      g.off_energy = (g.rows & SL_ENERGY) ? off : -1;
      off += (g.rows & SL_ENERGY) ? d->nt : 0;
      g.off_bound = (g.rows & SL_BOUND) ? off : -1;
      off += (g.rows & SL_BOUND) ? d->nt : 0;
      g.n_rows = off;
      g.p_rate = d->nx;
      g.p_c = (d->family == SNAP_FAMILY_B_BURGERS_BOUNDARY) ? d->nx + 1 : -1;
      g.n_params = d->nx + 1 + ((d->family == SNAP_FAMILY_B_BURGERS_BOUNDARY) ? d->nt : 0);
      p->info.n_vars = g.n_vars;
      p->info.n_rows_nominal = g.n_rows;
      p->info.n_params = g.n_params;
      p->info.n_blocks = d->nt;
      build_pattern_1d(p);
      break;
    }
    case SNAP_FAMILY_C_DIV_ENERGY: {
      if (d->nx < 4 || (d->nx & 1) || d->nx > 1024 || d->ny != d->nx) {
        free(p);
        return fail(SNAP_ERR_INVALID_ARG, "2-D grid must be square, even, in [4, 1024]");
      }
      if (!supported_2d(d->nx)) {
        free(p);
        return fail(SNAP_ERR_UNSUPPORTED, "2-D grid side must be even and at most 64 in this build");
      }
      const int N = d->nx;
      p->info.n_vars = 2 * N * N * d->nt;
      p->info.n_rows_nominal = N * N * d->nt + d->nt;
      p->info.n_params = 2;
      p->info.n_blocks = d->nt;
      build_pattern_2d(p, N, d->nt);
      cudaError_t e = setup_2d(p);
      if (e != cudaSuccess) {
        free(p->row_ptr); free(p->col_idx); free(p->active); free(p);
        return cuda_fail(e, "2-D setup");
      }
      break;
    }
    case SNAP_FAMILY_D_BURGERS_BC: {
      if (d->nx < 4 || d->nx > 65536 || d->rows != 0) {
        free(p);
        return fail(SNAP_ERR_INVALID_ARG, "family D: nx must be in [4, 65536] and rows 0");
      }
      p->info.n_vars = d->nx * d->nt;
      p->info.n_rows_nominal = 3 * d->nt;
      p->info.n_params = 2;
      p->info.n_blocks = d->nt;
      build_pattern_bc(p, d->nx, d->nt);
      break;
    }
    case SNAP_FAMILY_E_BURGERS_FLUX: {
      if (d->nx < 3 || d->nx > 512 || d->nt < 2 || d->rows != 0 || d->n_flux < 1 ||
          d->n_flux > d->nt - 1) {
        free(p);
        return fail(SNAP_ERR_INVALID_ARG,
                    "family E: nx in [3, 512], nt >= 2, 1 <= n_flux <= nt - 1, rows 0");
      }
      p->info.n_vars = d->nx * d->nt;
      p->info.n_rows_nominal = d->nx + d->nt + d->n_flux * d->nx;
      p->info.n_params = d->nx;
      p->info.n_blocks = d->nt - d->n_flux;
      build_pattern_flux(p, d->nx, d->nt, d->n_flux);
      break;
    }
    case SNAP_FAMILY_F_HEAT_ENERGY: {
      if (d->nx < 3 || d->nx > 512 || d->nt < 2 || d->rows != 0) {
        free(p);
        return fail(SNAP_ERR_INVALID_ARG, "family F: nx in [3, 512], nt >= 2, rows 0");
      }
      p->info.n_vars = d->nx * d->nt;
      p->info.n_rows_nominal = d->nx + d->nt + (d->nt - 1) * d->nx + (d->nt - 1);
      p->info.n_params = d->nx + 1;
      p->info.n_blocks = 1;
      build_pattern_heat(p, d->nx, d->nt);
      break;
    }
    case SNAP_FAMILY_TOY_LEFT_RIEMANN: {
      if (d->nx < 2 || d->nx > 4096) {
        free(p);
        return fail(SNAP_ERR_INVALID_ARG, "toy nx must be in [2, 4096]");
      }
      p->info.n_vars = d->nx * d->nt;
      p->info.n_params = d->nx;
      p->info.n_blocks = 1;
      build_pattern_toy(p, d->nx, d->nt);
      break;
    }
    default:
      free(p);
      return fail(SNAP_ERR_INVALID_ARG, "unknown family %d", d->family);
  }
  *out = p;
  return SNAP_OK;
}

void snap_problem_destroy(snap_problem_t p) {
  if (!p) return;
  if (p->desc.family == SNAP_FAMILY_C_DIV_ENERGY) teardown_2d(p);
  free(p->row_ptr);
  free(p->col_idx);
  free(p->active);
  free(p);
}

snap_status snap_problem_info(snap_problem_t p, snap_info *info) {
  if (!p || !info) return fail(SNAP_ERR_INVALID_ARG, "null argument");
  *info = p->info;
  return SNAP_OK;
}

snap_status snap_problem_pattern(snap_problem_t p, int *row_ptr, int *col_idx) {
  if (!p || !row_ptr || !col_idx) return fail(SNAP_ERR_INVALID_ARG, "null argument");
  memcpy(row_ptr, p->row_ptr, sizeof(int) * (size_t)(p->info.n_rows_nominal + 1));
  memcpy(col_idx, p->col_idx, sizeof(int) * (size_t)p->info.pattern_nnz);
  return SNAP_OK;
}

snap_status snap_problem_active_rows(snap_problem_t p, unsigned char *active) {
  if (!p || !active) return fail(SNAP_ERR_INVALID_ARG, "null argument");
  memcpy(active, p->active, (size_t)p->info.n_rows_nominal);
  return SNAP_OK;
}

snap_status snap_workspace_size(snap_problem_t p, int B, size_t *bytes) {
  if (!bytes) return fail(SNAP_ERR_INVALID_ARG, "null output");
  snap_status st = check_batch(p, B);
  if (st != SNAP_OK) return st;
  if (p->desc.family == SNAP_FAMILY_TOY_LEFT_RIEMANN) { *bytes = 0; return SNAP_OK; }
  *bytes = ws_bytes(p, B);
  return SNAP_OK;
}

snap_status snap_project(snap_problem_t p, int B, const double *u_hat, const double *params,
                         const double *u0, double *u, double *lambda, snap_stats *stats,
                         const snap_options *opt, void *workspace,
                         size_t workspace_bytes, snap_stream_t stream) {
  g_err[0] = 0;
  g_launches = 0;
  snap_status st = check_batch(p, B);
  if (st != SNAP_OK) return st;
  if (p->desc.family == SNAP_FAMILY_TOY_LEFT_RIEMANN)
    return fail(SNAP_ERR_UNSUPPORTED, "the toy family supports pattern queries only");
  snap_options o;
  snap_options_default(&o);
  if (opt) o = *opt;
  if ((st = check_opts(o)) != SNAP_OK) return st;
  if (B == 0) return SNAP_OK;
  if (!u_hat || !params || !u || !lambda)
    return fail(SNAP_ERR_INVALID_ARG, "null u_hat / params / u / lambda");
  if (!aligned16(u_hat) || !aligned16(u) || (u0 && !aligned16(u0)))
    return fail(SNAP_ERR_INVALID_ARG, "u_hat, u0 and u must be 16-byte aligned");
  if (u == u_hat || u == u0 || (double *)lambda == u)
    return fail(SNAP_ERR_INVALID_ARG, "outputs may not alias inputs");
  const size_t need = ws_bytes(p, B);
  if (need > 0 && (!workspace || workspace_bytes < need))
    return fail(SNAP_ERR_WORKSPACE, "workspace of %zu bytes required (got %zu)", need, workspace_bytes);
  int path = o.path;
  if ((path == SNAP_PATH_MOMENT || path == SNAP_PATH_MIXED) && u0 && u0 != u_hat)
    return fail(SNAP_ERR_UNSUPPORTED, "the moment paths need u0 = u_hat");
  if (path == SNAP_PATH_AUTO) path = (u0 && u0 != u_hat) ? SNAP_PATH_GENERAL : SNAP_PATH_MIXED;
  if (u0 == u_hat) u0 = nullptr;
  const SolverOpts so = to_solver(o);
  cudaError_t e;
  if (p->desc.family == SNAP_FAMILY_F_HEAT_ENERGY) {
    if (u0) return fail(SNAP_ERR_UNSUPPORTED, "family F starts at u_hat (square active rows)");
    e = launch_heat_forward(p, B, u_hat, params, u, lambda, stats, o.tol_h, (cudaStream_t)stream);
  } else if (p->desc.family == SNAP_FAMILY_D_BURGERS_BC) {
    if (u0) return fail(SNAP_ERR_UNSUPPORTED, "family D starts at u_hat (linear rows: one step)");
    e = launch_1dbc_forward(p, B, u_hat, params, u, lambda, stats, so, workspace,
                            (cudaStream_t)stream);
  } else if (p->desc.family == SNAP_FAMILY_E_BURGERS_FLUX) {
    if (u0) return fail(SNAP_ERR_UNSUPPORTED, "family E starts at u_hat (direct evaluation)");
    e = launch_1dflux_forward(p, B, u_hat, params, u, lambda, stats, so, workspace,
                              (cudaStream_t)stream);
  } else if (p->desc.family == SNAP_FAMILY_C_DIV_ENERGY)
    e = launch_2d_forward(p, B, u_hat, params, u0, u, lambda, stats, so, path, workspace,
                          (cudaStream_t)stream);
  else
    e = launch_1d_forward(p, B, u_hat, params, u0, u, lambda, stats, so, path, workspace,
                          (cudaStream_t)stream);
  if (e == cudaErrorNotSupported) return fail(SNAP_ERR_UNSUPPORTED, "unsupported request for this family");
  if (e != cudaSuccess) return cuda_fail(e, "snap_project launch");
  return SNAP_OK;
}

snap_status snap_project_backward(snap_problem_t p, int B, const double *grad_u,
                                  const double *u, const double *lambda, const double *params,
                                  const snap_stats *stats, double *grad_u_hat,
                                  double *grad_params, void *workspace,
                                  size_t workspace_bytes, snap_stream_t stream) {
  g_err[0] = 0;
  g_launches = 0;
  snap_status st = check_batch(p, B);
  if (st != SNAP_OK) return st;
  if (p->desc.family == SNAP_FAMILY_TOY_LEFT_RIEMANN)
    return fail(SNAP_ERR_UNSUPPORTED, "the toy family supports pattern queries only");
  if (B == 0) return SNAP_OK;
  if (!grad_u || !u || !lambda || !params || !grad_u_hat)
    return fail(SNAP_ERR_INVALID_ARG, "null grad_u / u / lambda / params / grad_u_hat");
  if (!aligned16(grad_u) || !aligned16(u) || !aligned16(grad_u_hat))
    return fail(SNAP_ERR_INVALID_ARG, "grad_u, u and grad_u_hat must be 16-byte aligned");
  if (grad_u_hat == grad_u || grad_u_hat == u || (grad_params && grad_params == params))
    return fail(SNAP_ERR_INVALID_ARG, "outputs may not alias inputs");
  const size_t need = ws_bytes(p, B);
  if (need > 0 && (!workspace || workspace_bytes < need))
    return fail(SNAP_ERR_WORKSPACE, "workspace of %zu bytes required (got %zu)", need, workspace_bytes);
  cudaError_t e;
  if (p->desc.family == SNAP_FAMILY_F_HEAT_ENERGY)
    e = launch_heat_backward(p, B, grad_u, u, params, stats, grad_u_hat, grad_params,
                             (cudaStream_t)stream);
  else if (p->desc.family == SNAP_FAMILY_D_BURGERS_BC)
    e = launch_1dbc_backward(p, B, grad_u, stats, grad_u_hat, grad_params, workspace,
                             (cudaStream_t)stream);
  else if (p->desc.family == SNAP_FAMILY_E_BURGERS_FLUX)
    e = launch_1dflux_backward(p, B, grad_u, u, stats, grad_u_hat, grad_params, workspace,
                               (cudaStream_t)stream);
  else if (p->desc.family == SNAP_FAMILY_C_DIV_ENERGY)
    e = launch_2d_backward(p, B, grad_u, u, lambda, params, stats, grad_u_hat, grad_params,
                           workspace, (cudaStream_t)stream);
  else
    e = launch_1d_backward(p, B, grad_u, u, lambda, params, stats, grad_u_hat, grad_params,
                           workspace, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "snap_project_backward launch");
  return SNAP_OK;
}

snap_status snap_constraint_residual(snap_problem_t p, int B, const double *u,
                                     const double *params, double *h, double *h_inf,
                                     void *workspace, size_t workspace_bytes,
                                     snap_stream_t stream) {
  g_err[0] = 0;
  g_launches = 0;
  snap_status st = check_batch(p, B);
  if (st != SNAP_OK) return st;
  if (p->desc.family == SNAP_FAMILY_TOY_LEFT_RIEMANN)
    return fail(SNAP_ERR_UNSUPPORTED, "the toy family supports pattern queries only");
  if (B == 0) return SNAP_OK;
  if (!u || !params) return fail(SNAP_ERR_INVALID_ARG, "null u / params");
  const size_t need = ws_bytes(p, B);
  if (need > 0 && (!workspace || workspace_bytes < need))
    return fail(SNAP_ERR_WORKSPACE, "workspace of %zu bytes required (got %zu)", need, workspace_bytes);
  cudaError_t e;
  if (p->desc.family == SNAP_FAMILY_F_HEAT_ENERGY)
    e = launch_heat_residual(p, B, u, params, h, h_inf, (cudaStream_t)stream);
  else if (p->desc.family == SNAP_FAMILY_D_BURGERS_BC)
    e = launch_1dbc_residual(p, B, u, params, h, h_inf, workspace, (cudaStream_t)stream);
  else if (p->desc.family == SNAP_FAMILY_E_BURGERS_FLUX)
    e = launch_1dflux_residual(p, B, u, params, h, h_inf, workspace, (cudaStream_t)stream);
  else if (p->desc.family == SNAP_FAMILY_C_DIV_ENERGY)
    e = launch_2d_residual(p, B, u, params, h, h_inf, workspace, (cudaStream_t)stream);
  else
    e = launch_1d_residual(p, B, u, params, h, h_inf, workspace, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "snap_constraint_residual launch");
  return SNAP_OK;
}

}  // extern "C"

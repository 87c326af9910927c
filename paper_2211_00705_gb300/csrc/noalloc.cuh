// One explicit time step for callers that cannot allocate GPU memory (imexds_step_uniform_noalloc).
// Included once, from imexds.cu. The scratch this step needs (per-instance offsets, widths, time steps
// and wave-speed maxima) lives in one file-scope device array instead of memory allocated by a context.
#pragma once

namespace imexds_noalloc {

constexpr int kMaxInst = 16384;  // largest batch the fixed scratch holds

struct Scratch {
  int n_lattice[kMaxInst];
  int lat_off[kMaxInst + 1];
  int tile_off[kMaxInst + 1];
  double x_left[kMaxInst];
  double x_right[kMaxInst];
  double h[kMaxInst];
  double dt[kMaxInst];
  int err;  // set by k_dt: kErrMixed, kErrState (bits)
};

constexpr int kErrMixed = 1;  // an instance holds cells of both phases
constexpr int kErrState = 2;  // a phase byte above 1, a density that is not positive and finite, or a non-finite m

// The scratch array (about 0.7 MB); every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) Scratch g_scratch;

// Offsets of the packed cell arrays and of the 32-cell tiles, widths h = (x_R - x_L) / N.
__global__ void k_setup(Scratch* s, int n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int lo = 0, to = 0;
    for (int i = 0; i < n; ++i) {
      s->lat_off[i] = lo;
      s->tile_off[i] = to;
      lo += s->n_lattice[i];
      to += (s->n_lattice[i] + 31) >> 5;
      s->h[i] = (s->x_right[i] - s->x_left[i]) / (double)s->n_lattice[i];
    }
    s->lat_off[n] = lo;
    s->tile_off[n] = to;
    s->err = 0;
  }
}

// Time step of each instance from the CFL condition (Eq. cfl_cond:unif): dt = C h / max_i(|u_i| + a). The
// inputs are device arrays that no host code has seen, so this kernel also checks them: a phase byte above 1,
// a density that is not positive and finite or a non-finite momentum sets kErrState, and an instance with
// cells of both phases sets kErrMixed. A phase is only used as an index after masking it to 0 or 1.
__global__ void k_dt(Scratch* s, Fluid F, double cfl, const double* rho, const double* m, const uint8_t* ph,
                     double* dt_out) {
  const int i = blockIdx.x;
  const int o = s->lat_off[i], N = s->n_lattice[i];
  const int p0 = ph[o];
  double S = 0.0;
  int mixed = 0, bad = 0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const int pj = ph[o + j];
    const double r = rho[o + j], mm = m[o + j];
    const bool ok = pj <= 1 && r > 0.0 && isfinite(r) && isfinite(mm);
    bad |= ok ? 0 : 1;
    mixed |= (pj != p0);
    if (ok) S = fmax(S, fabs(div_nr(mm, r)) + F.ph[pj & 1].a);
  }
  __shared__ double red[32];
  __shared__ int any_mixed, any_bad;
  if (threadIdx.x == 0) {
    any_mixed = 0;
    any_bad = 0;
  }
  for (int off = 16; off > 0; off >>= 1) S = fmax(S, __shfl_down_sync(0xffffffffu, S, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = S;
  if (mixed) atomicOr(&any_mixed, 1);
  if (bad) atomicOr(&any_bad, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    double Sx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) Sx = fmax(Sx, red[w]);
    double dt = cfl * s->h[i] / Sx;
    s->dt[i] = dt;
    dt_out[i] = dt;
    if (any_mixed) atomicOr(&s->err, kErrMixed);
    if (any_bad) atomicOr(&s->err, kErrState);
  }
}

// The explicit HLL sweep of the library for cells away from any phase boundary: HLL fluxes and the
// explicit update, one warp per 32-cell tile (the same arithmetic as the library's sweep). Launched after
// k_dt on the same stream; it writes nothing when k_dt found bad input.
__global__ void k_sweep(const Scratch* s, Fluid F, int n, int n_tiles, const double* rho, const double* m,
                        const uint8_t* ph, double* rho_out, double* m_out) {
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (t >= n_tiles || s->err) return;
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = n - 1;  // instance holding tile t
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (s->tile_off[mid] <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int i = lo, o = s->lat_off[i], N = s->n_lattice[i];
  const int j0 = (t - s->tile_off[i]) << 5;
  const Phase& E = F.ph[ph[o] & 1];
  auto load = [&](int j, double& r, double& mm, double& u, double& f1) {
    r = rho[o + j];
    mm = m[o + j];
    u = div_nr(mm, r);
    f1 = __fma_rn(mm, u, pressure_fma(E, r));
  };
  const int j = j0 + lane;
  double r = 1.0, mm = 0.0, u = 0.0, f1 = 0.0;
  if (j < N) load(j, r, mm, u, f1);
  double rl = __shfl_up_sync(0xffffffffu, r, 1), ml = __shfl_up_sync(0xffffffffu, mm, 1);
  double ul = __shfl_up_sync(0xffffffffu, u, 1), fl1 = __shfl_up_sync(0xffffffffu, f1, 1);
  if (lane == 0 && j0 > 0) load(j0 - 1, rl, ml, ul, fl1);
  // flux at the left face of cell j (transmissive at the domain ends)
  double F0 = 0.0, F1 = 0.0;
  if (j <= N) {
    if (j == 0) {
      F0 = mm;
      F1 = f1;
    } else if (j == N) {
      F0 = ml;
      F1 = fl1;
    } else {
      hll_pre(E.a, rl, ml, ul, fl1, r, mm, u, f1, F0, F1);
    }
  }
  double G0 = __shfl_down_sync(0xffffffffu, F0, 1), G1 = __shfl_down_sync(0xffffffffu, F1, 1);
  if (lane == 31 && j < N) {
    if (j + 1 == N) {
      G0 = mm;
      G1 = f1;
    } else {
      double rr, mr, ur, fr1;
      load(j + 1, rr, mr, ur, fr1);
      hll_pre(E.a, r, mm, u, f1, rr, mr, ur, fr1, G0, G1);
    }
  }
  if (j < N) {
    const double lam = s->dt[i] / s->h[i];
    rho_out[o + j] = __fma_rn(-lam, G0 - F0, r);
    m_out[o + j] = __fma_rn(-lam, G1 - F1, mm);
  }
}

}  // namespace imexds_noalloc

// det.cu -- the deterministic orbit deposit (option deterministic_deposit).
//
// The particle map deposits q vbar Sbar / dV (Eq. orbit-current-energy) with
// FP64 atomics, so the order in which a node's contributions are summed, and
// the last bits of the sum, change from run to run and differ between nodes
// that receive equal contributions.  This path instead computes every node's
// current in one thread, over the particles whose orbits can reach it, in an
// order fixed by their cell (a fixed scan of the neighbouring cells) and,
// within a cell, by their offset and then their load index.  The sum is then
// the same from run to run, and nodes whose neighbourhoods hold equal
// particle configurations receive bitwise equal currents.  Each particle's
// orbit weight for the node is recomputed (the knot-split walk and its
// Gauss-Legendre points, restricted to the one node), so the pass costs
// several times the atomic deposit: it is a checking mode.
#include "map_device.cuh"

namespace {

// particles per cell (cell = nearest node)
__global__ void k_det_count(int64_t np, int64_t cap, const int32_t *__restrict__ cell, int dim,
                            int n0, int n01, int32_t *count) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  int key = cell[i];
  if (dim > 1) key += n0 * cell[cap + i];
  if (dim > 2) key += n01 * cell[2 * cap + i];
  atomicAdd(count + key, 1);
}

// exclusive prefix sum of the counts (one block), start[Ng] = total
__global__ void k_det_scan(const int32_t *__restrict__ count, int32_t *start, int Ng) {
  __shared__ int32_t carry;
  __shared__ int32_t part[1024];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < Ng; base += 1024) {
    const int g = base + threadIdx.x;
    part[threadIdx.x] = g < Ng ? count[g] : 0;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan in shared memory
      const int32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    if (g < Ng) start[g] = carry + part[threadIdx.x] - count[g];
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) start[Ng] = carry;
}

// scatter particle indices into their cell's range (order still arbitrary)
__global__ void k_det_fill(int64_t np, int64_t cap, const int32_t *__restrict__ cell, int dim,
                           int n0, int n01, const int32_t *__restrict__ start, int32_t *cursor,
                           int32_t *list) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  int key = cell[i];
  if (dim > 1) key += n0 * cell[cap + i];
  if (dim > 2) key += n01 * cell[2 * cap + i];
  list[start[key] + atomicAdd(cursor + key, 1)] = (int32_t)i;
}

// order within a cell: by offset (x, then y, then z), then by load index
__device__ __forceinline__ bool det_before(int a, int b, const double *off, int64_t cap, int dim,
                                           const int64_t *id) {
  for (int l = 0; l < dim; l++) {
    const double oa = off[l * cap + a], ob = off[l * cap + b];
    if (oa != ob) return oa < ob;
  }
  return id[a] < id[b];
}

__global__ void k_det_order(const int32_t *__restrict__ start, int32_t *list, int Ng,
                            const double *__restrict__ off, int64_t cap, int dim,
                            const int64_t *__restrict__ id) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Ng) return;
  const int b = start[g], e = start[g + 1];
  for (int k = b + 1; k < e; k++) {  // insertion sort: cells hold tens of particles
    const int v = list[k];
    int m = k - 1;
    while (m >= b && det_before(v, list[m], off, cap, dim, id)) {
      list[m + 1] = list[m];
      m--;
    }
    list[m + 1] = v;
  }
}

// reach of the deposit in cells: the largest base shift of an orbit piece,
// floor(1 + |vbar dt / dx|), over particles and dimensions
__global__ void k_det_reach(int64_t np, int64_t cap, int dim, const double *__restrict__ vbar,
                            PGeom pg, double dt, int *reach) {  // dt = 0: point deposits
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  int r = 1;
  for (int l = 0; l < dim; l++) {
    const double d = fabs(vbar[l * cap + i] * dt * pg.inv_dx[l]);
    const int rl = isfinite(d) && d < 64.0 ? (int)floor(1.0 + d) : 64;
    r = rl > r ? rl : r;
  }
  atomicMax(reach, r);
}

// One node's orbit-averaged weight from one particle: the walk's pieces that
// put the node in their 3^D stencil, each integrated at its Gauss-Legendre
// points exactly as DepositOrbit integrates it.
template <int D>
struct NodeDot {
  const KConst<double> *kc;
  int order;
  double off[3], del[3];
  int t[3];   // the node relative to the particle's nearest node
  double S;
  __device__ __forceinline__ void operator()(const int base[3], double sa, double sb) {
    int r[3] = {0, 0, 0};
    for (int l = 0; l < D; l++) {
      r[l] = t[l] - base[l];
      if (r[l] < -1 || r[l] > 1) return;
    }
    if (D == 3) {
      PieceAcc<2, double> pa;
      double Wz[9], W1z[9];
      accumulate_slab<double, false>(*kc, off, del, base, sa, sb, r[2] + 1, pa, Wz, W1z, order);
      S += pa.Sb[(r[0] + 1) + 3 * (r[1] + 1)];
    } else {
      PieceAcc<D, double> pa;
      accumulate_piece<D, double, false>(*kc, off, del, base, sa, sb, pa, order);
      S += pa.Sb[(r[0] + 1) + (D > 1 ? 3 * (r[1] + 1) : 0)];
    }
  }
};

// One thread per node: J_c(g) = sum over the cells within the reach (a fixed
// scan order) and their particles (list order) of q vbar_c Sbar(g) / dV.
// With dt = 0 the orbits have zero length and this is the point deposit of
// pic_start (the Gauss-Legendre weights sum to one); rho, if given, then
// receives sum q S / dV on top of its contents.
template <int D>
__global__ void k_det_gather(int Ng, PGeom pg, KConst<double> kc, double dt, int order,
                             int64_t cap, const int32_t *__restrict__ cell,
                             const double *__restrict__ off, const double *__restrict__ vbar,
                             const double *__restrict__ w, const int32_t *__restrict__ sp,
                             const int32_t *__restrict__ start, const int32_t *__restrict__ list,
                             const int *__restrict__ reach, double *__restrict__ J,
                             double *__restrict__ rho, EvalCounters *__restrict__ cnt) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Ng) return;
  // an orbit piece's base shifts by at most `reach` cells and its stencil
  // reaches one node further
  const int R = *reach + 1;
  int gc[3] = {g % pg.n[0], D > 1 ? (g / pg.n[0]) % pg.n[1] : 0, D > 2 ? g / pg.n01 : 0};
  for (int l = 0; l < D; l++)
    if (2 * R + 1 > pg.n[l]) {  // the stencil would alias periodic images
      if (g == 0) atomicOr(&cnt->status, PIC_ST_PIECES);
      for (int c = 0; c < 3; c++) J[(size_t)c * Ng + g] = 0.0;
      return;
    }
  double acc[3] = {0.0, 0.0, 0.0}, charge = 0.0;
  const int Rz = D > 2 ? R : 0, Ry = D > 1 ? R : 0;
  for (int dz = -Rz; dz <= Rz; dz++)
    for (int dy = -Ry; dy <= Ry; dy++)
      for (int dx = -R; dx <= R; dx++) {
        const int d[3] = {dx, dy, dz};
        int c = 0;
        for (int l = 0; l < D; l++) {
          const int cl = (gc[l] + d[l]) & pg.mask[l];
          c += l == 0 ? cl : (l == 1 ? pg.n0 * cl : pg.n01 * cl);
        }
        for (int k = start[c]; k < start[c + 1]; k++) {
          const int i = list[k];
          NodeDot<D> nd;
          nd.kc = &kc;
          nd.order = order;
          nd.S = 0.0;
          double vb[3];
          for (int l = 0; l < 3; l++) {
            vb[l] = vbar[l * cap + i];
            nd.off[l] = l < D ? off[l * cap + i] : 0.0;
            nd.del[l] = l < D ? vb[l] * dt * kc.inv_dx[l] : 0.0;
            nd.t[l] = l < D ? -d[l] : 0;
          }
          walk_orbit<D, double>(nd.off, nd.del, nd, order);
          const double qs = w[i] * kc.qs[sp[i]] * kc.inv_dV * nd.S;
          for (int l = 0; l < 3; l++) acc[l] += qs * vb[l];
          charge += qs;
        }
      }
  for (int l = 0; l < 3; l++) J[(size_t)l * Ng + g] = acc[l];
  if (rho) rho[g] += charge;
}

// mechanical velocity v = p / (m gamma), p = P - q A_h(x), in slot order
template <int D>
__global__ void k_det_point_velocity(int64_t np, int64_t cap, const int32_t *__restrict__ cell_a,
                                     const double *__restrict__ off_a,
                                     const double *__restrict__ P, const double *__restrict__ w,
                                     const int32_t *__restrict__ sp, const double *__restrict__ A,
                                     PGeom pg, KConst<double> kc, double *v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  int cell[3] = {0, 0, 0};
  double off[3] = {0.0, 0.0, 0.0};
  for (int l = 0; l < D; l++) {
    cell[l] = cell_a[l * cap + i];
    off[l] = off_a[l * cap + i];
  }
  double Ax[3];
  point_interp<D, double>(pg, cell, off, A, Ax);
  const int s = sp[i];
  const double q = w[i] * kc.qs[s], m = w[i] * kc.ms[s];
  double p[3], p2 = 0.0;
  for (int c = 0; c < 3; c++) {
    p[c] = P[c * cap + i] - q * Ax[c];
    p2 += p[c] * p[c];
  }
  const double gam = sqrt(1.0 + p2 / (m * m * kc.kappa * kc.kappa));
  for (int c = 0; c < 3; c++) v[c * cap + i] = p[c] / (m * gam);
}

}  // namespace

int det_alloc(pic_ctx *ctx) {
  if (!ctx->opt.deterministic_deposit) return PIC_OK;
  const size_t Ng = ctx->g.Ng;
  if (!ctx->det_count) {
    CK(cudaMalloc((void **)&ctx->det_count, sizeof(int32_t) * Ng));
    CK(cudaMalloc((void **)&ctx->det_cursor, sizeof(int32_t) * Ng));
    CK(cudaMalloc((void **)&ctx->det_start, sizeof(int32_t) * (Ng + 1)));
    CK(cudaMalloc((void **)&ctx->det_reach, sizeof(int)));
  }
  if (ctx->det_cap < ctx->cap) {
    if (ctx->det_list) cudaFree(ctx->det_list);
    ctx->det_list = nullptr;
    CK(cudaMalloc((void **)&ctx->det_list, sizeof(int32_t) * ctx->cap));
    ctx->det_cap = ctx->cap;
  }
  return PIC_OK;
}

void det_free(pic_ctx *ctx) {
  int32_t *p[] = {ctx->det_count, ctx->det_cursor, ctx->det_start, ctx->det_list};
  for (int32_t *q : p)
    if (q) cudaFree(q);
  if (ctx->det_reach) cudaFree(ctx->det_reach);
  ctx->det_count = ctx->det_cursor = ctx->det_start = ctx->det_list = nullptr;
  ctx->det_reach = nullptr;
  ctx->det_cap = 0;
}

namespace {

// per-cell particle lists in the fixed order (offset, then load index)
int det_lists(pic_ctx *ctx) {
  const Geom &g = ctx->g;
  const int Ng = g.Ng, d = g.dim;
  const int64_t np = ctx->np, cap = ctx->cap;
  CK(cudaMemsetAsync(ctx->det_count, 0, sizeof(int32_t) * Ng, ctx->st));
  CK(cudaMemsetAsync(ctx->det_cursor, 0, sizeof(int32_t) * Ng, ctx->st));
  if (np > 0) {
    k_det_count<<<nblk(np), kPT, 0, ctx->st>>>(np, cap, ctx->cell, d, g.n[0], g.n[0] * g.n[1],
                                               ctx->det_count);
    KCHECK();
  }
  k_det_scan<<<1, 1024, 0, ctx->st>>>(ctx->det_count, ctx->det_start, Ng);
  KCHECK();
  if (np > 0) {
    k_det_fill<<<nblk(np), kPT, 0, ctx->st>>>(np, cap, ctx->cell, d, g.n[0], g.n[0] * g.n[1],
                                              ctx->det_start, ctx->det_cursor, ctx->det_list);
    KCHECK();
    k_det_order<<<(Ng + 127) / 128, 128, 0, ctx->st>>>(ctx->det_start, ctx->det_list, Ng,
                                                       (const double *)ctx->off, cap, d, ctx->id);
    KCHECK();
  }
  return PIC_OK;
}

__global__ void k_det_slots(int64_t np, const int32_t *__restrict__ list, int64_t *slot) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < np) slot[list[k]] = k;
}

// cell lists, reach and the node gather for velocities vel (3 x cap) and
// orbit duration dt (0: point deposit)
int det_run(pic_ctx *ctx, double *J, double *rho, const double *vel, double dt,
            const StepConst &sc) {
  const Geom &g = ctx->g;
  const int Ng = g.Ng, d = g.dim;
  const int64_t np = ctx->np, cap = ctx->cap;
  if (!ctx->det_count || ctx->det_cap < cap) {
    ctx->err = "deterministic deposit: buffers not allocated (pic_start first)";
    return PIC_ESTATE;
  }
  const PGeom pg = pgeom(ctx);
  int e;
  if ((e = det_lists(ctx))) return e;
  CK(cudaMemsetAsync(ctx->det_reach, 0, sizeof(int), ctx->st));
  if (np > 0) {
    k_det_reach<<<nblk(np), kPT, 0, ctx->st>>>(np, cap, d, vel, pg, dt, ctx->det_reach);
    KCHECK();
  }
  const KConst<double> kc = kconst<double>(sc, pg);
  const int nb = (Ng + 127) / 128;
#define PIC_DET(DD)                                                                           \
  k_det_gather<DD><<<nb, 128, 0, ctx->st>>>(Ng, pg, kc, dt, ctx->opt.order, cap, ctx->cell,    \
                                            (const double *)ctx->off, vel, ctx->w, ctx->sp,    \
                                            ctx->det_start, ctx->det_list, ctx->det_reach, J,  \
                                            rho, ctx->cnt_dev)
  if (d == 1) PIC_DET(1);
  else if (d == 2) PIC_DET(2);
  else PIC_DET(3);
#undef PIC_DET
  KCHECK();
  return PIC_OK;
}

}  // namespace

// Recompute the orbit current of the last map evaluation (from the particles'
// vbar) deterministically into J, overwriting it.  Queues work only.
int det_deposit(pic_ctx *ctx, double *J, const StepConst &sc) {
  return det_run(ctx, J, nullptr, (const double *)ctx->vbar, ctx->dt, sc);
}

// The point deposits of pic_start: rho += sum q S(x) / dV (rho holds the
// background), J = sum q v S(x) / dV with v = p / (m gamma), both in a fixed
// order.  Uses the context's export scratch for v.
int det_point_deposit(pic_ctx *ctx, double *rho, double *J, const StepConst &sc) {
  const int64_t np = ctx->np, cap = ctx->cap;
  double *v = ctx->tmp_d;  // 7 * cap doubles
  if (np > 0) {
    const PGeom pg = pgeom(ctx);
    const KConst<double> kc = kconst<double>(sc, pg);
#define PIC_PV(DD)                                                                           \
  k_det_point_velocity<DD><<<nblk(np), kPT, 0, ctx->st>>>(                                 \
      np, cap, ctx->cell, (const double *)ctx->off, (const double *)ctx->P, ctx->w, ctx->sp, \
      ctx->A_real, pg, kc, v)
    if (ctx->g.dim == 1) PIC_PV(1);
    else if (ctx->g.dim == 2) PIC_PV(2);
    else PIC_PV(3);
#undef PIC_PV
    KCHECK();
  }
  return det_run(ctx, J, rho, v, 0.0, sc);
}

// The counting sort's destination slots in the lists' fixed order (so the
// particle order after a sort, and every reduction over it, does not depend
// on the order of atomic operations).
int det_sort_slots(pic_ctx *ctx, int64_t *slot) {
  if (!ctx->det_count || ctx->det_cap < ctx->cap) {
    ctx->err = "deterministic deposit: buffers not allocated (pic_start first)";
    return PIC_ESTATE;
  }
  int e;
  if ((e = det_lists(ctx))) return e;
  if (ctx->np > 0) {
    k_det_slots<<<nblk(ctx->np), kPT, 0, ctx->st>>>(ctx->np, ctx->det_list, slot);
    KCHECK();
  }
  return PIC_OK;
}

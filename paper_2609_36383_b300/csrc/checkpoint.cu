// checkpoint.cu -- pic_checkpoint_*: the accepted state of a context as one
// byte image (a fixed header followed by raw sections), for checkpoint and
// exact resume.
//
// pic_set_state restores a state from the real-space arrays a user reads
// with pic_get_*; those pass through an inverse and a forward FFT, so a run
// resumed that way agrees with the uninterrupted run to rounding only.  The
// image instead holds the device arrays themselves: the particles in their
// storage (slot) order with their cell/offset split, and the potentials as
// the spectral coefficients the field step advances.  Loading it into a
// context of the same mesh, precision and species gives that context the
// very bits the saving context had, so the next steps repeat the
// uninterrupted run exactly wherever the run itself is reproducible (the
// deterministic deposit; the atomic deposit reorders its sums from run to
// run).
//
// Everything an image says is checked on the host before anything reaches
// the device: a checksum over the payload, the sizes, and every value used
// as an index (cells inside the mesh, offsets inside a cell, species in
// range, load-order indices a permutation), so a damaged or foreign image is
// refused with PIC_EARG and never becomes an out-of-range access.
#include "pic_internal.cuh"
#include "trace.cuh"

#include <cmath>
#include <cstring>
#include <vector>

namespace {

static_assert(sizeof(pic_checkpoint_header) == 256, "checkpoint header layout");

constexpr char kMagic[8] = {'P', 'I', 'C', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kVersion = 1;

// FNV-1a, 64-bit (Fowler, Noll, Vo): offset basis and prime of the
// published definition
uint64_t fnv1a64(const unsigned char *p, uint64_t n) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (uint64_t i = 0; i < n; i++) {
    h ^= p[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

uint64_t round16(uint64_t b) { return (b + 15) & ~uint64_t(15); }

// byte offsets of the payload sections, in image order
struct Layout {
  enum { CELL, OFF, P, W, SP, ID, PHI, PSI, RHO, A, U, AREAL, JACC, NSEC };
  uint64_t off[NSEC + 1];
};

Layout layout(int dim, int rsize, int64_t np, int64_t Ng) {
  const uint64_t n = (uint64_t)np, g = (uint64_t)Ng;
  const uint64_t bytes[Layout::NSEC] = {
      4 * dim * n,        // cell    int32 [dim][np]
      rsize * dim * n,    // off     real  [dim][np]
      rsize * 3 * n,      // P       real  [3][np]
      8 * n,              // w       f64   [np]
      4 * n,              // sp      int32 [np]
      8 * n,              // id      int64 [np]
      16 * g,             // phi     c128  [Ng]
      16 * g,             // psi     c128  [Ng]
      16 * g,             // rho     c128  [Ng]
      16 * 3 * g,         // A       c128  [3][Ng]
      16 * 3 * g,         // U       c128  [3][Ng]
      8 * 3 * g,          // A real  f64   [3][Ng]
      8 * 3 * g};         // J acc.  f64   [3][Ng]
  Layout L;
  uint64_t o = sizeof(pic_checkpoint_header);
  for (int s = 0; s < Layout::NSEC; s++) {
    L.off[s] = o;
    o += round16(bytes[s]);
  }
  L.off[Layout::NSEC] = o;
  return L;
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

template <typename T>
bool offsets_ok(const unsigned char *p, uint64_t count) {
  for (uint64_t i = 0; i < count; i++) {
    T v;
    std::memcpy(&v, p + i * sizeof(T), sizeof(T));
    if (!(v >= T(-0.5) && v <= T(0.5))) return false;  // also rejects NaN
  }
  return true;
}

// The whole validation of an image, host only.  On failure returns false and
// points *why at the reason.
bool check_image(const void *image, uint64_t bytes, pic_checkpoint_header *hdr_out,
                 const char **why) {
  if (!image || bytes < sizeof(pic_checkpoint_header)) {
    *why = "checkpoint image shorter than its header";
    return false;
  }
  const unsigned char *b = (const unsigned char *)image;
  pic_checkpoint_header h;
  std::memcpy(&h, b, sizeof h);
  if (std::memcmp(h.magic, kMagic, 8) != 0) {
    *why = "not a checkpoint image (magic)";
    return false;
  }
  if (h.version != kVersion || h.header_bytes != sizeof(pic_checkpoint_header)) {
    *why = "checkpoint image of another format version";
    return false;
  }
  if (h.total_bytes != bytes) {
    *why = "checkpoint image truncated or padded (size differs from its header)";
    return false;
  }
  if (h.dim < 1 || h.dim > 3) {
    *why = "checkpoint header: bad dimension";
    return false;
  }
  int64_t Ng = 1;
  for (int l = 0; l < 3; l++) {
    if (l < h.dim ? !pow2_in(h.n[l], 4, 4096) : h.n[l] != 1) {
      *why = "checkpoint header: bad mesh size";
      return false;
    }
    Ng *= h.n[l];
  }
  if ((h.precision != PIC_FP64 && h.precision != PIC_MIXED) || h.nspecies < 1 ||
      h.nspecies > PIC_MAX_SPECIES || h.np < 0 || h.np > (int64_t(1) << 40) ||
      h.steps_done < 0 || h.sort_every < 0) {
    *why = "checkpoint header: bad precision, species count, particle count or counters";
    return false;
  }
  const int rsize = h.precision == PIC_FP64 ? 8 : 4;
  const Layout L = layout(h.dim, rsize, h.np, Ng);
  if (L.off[Layout::NSEC] != bytes) {
    *why = "checkpoint image size does not match its header";
    return false;
  }
  if (fnv1a64(b + sizeof h, bytes - sizeof h) != h.checksum) {
    *why = "checkpoint payload checksum mismatch";
    return false;
  }
  // every value later used as an index
  const uint64_t n = (uint64_t)h.np;
  for (int l = 0; l < h.dim; l++) {
    const unsigned char *c = b + L.off[Layout::CELL] + 4 * l * n;
    for (uint64_t i = 0; i < n; i++) {
      int32_t v;
      std::memcpy(&v, c + 4 * i, 4);
      if (v < 0 || v >= h.n[l]) {
        *why = "checkpoint: particle cell outside the mesh";
        return false;
      }
    }
  }
  const unsigned char *o = b + L.off[Layout::OFF];
  if (!(rsize == 8 ? offsets_ok<double>(o, h.dim * n) : offsets_ok<float>(o, h.dim * n))) {
    *why = "checkpoint: particle offset outside [-1/2, 1/2] of a cell";
    return false;
  }
  for (uint64_t i = 0; i < n; i++) {
    int32_t s;
    std::memcpy(&s, b + L.off[Layout::SP] + 4 * i, 4);
    if (s < 0 || s >= h.nspecies) {
      *why = "checkpoint: species index out of range";
      return false;
    }
  }
  std::vector<unsigned char> seen(n, 0);
  for (uint64_t i = 0; i < n; i++) {
    int64_t id;
    std::memcpy(&id, b + L.off[Layout::ID] + 8 * i, 8);
    if (id < 0 || (uint64_t)id >= n || seen[id]) {
      *why = "checkpoint: load-order indices are not a permutation";
      return false;
    }
    seen[id] = 1;
  }
  if (hdr_out) *hdr_out = h;
  return true;
}

// the checkpoint header this context's state would get (checksum and size
// left for the caller)
pic_checkpoint_header header_of(const pic_ctx *ctx) {
  pic_checkpoint_header h;
  std::memset(&h, 0, sizeof h);
  std::memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.header_bytes = sizeof h;
  h.dim = ctx->g.dim;
  for (int l = 0; l < 3; l++) {
    h.n[l] = ctx->g.n[l];
    h.L[l] = ctx->g.L[l];
    h.x0[l] = ctx->g.x0[l];
  }
  h.precision = ctx->rsize == 8 ? PIC_FP64 : PIC_MIXED;
  h.nspecies = ctx->nspecies;
  h.sort_every = ctx->opt.sort_every;
  for (int s = 0; s < PIC_MAX_SPECIES; s++) {
    h.q[s] = s < ctx->nspecies ? ctx->qs[s] : 0.0;
    h.m[s] = s < ctx->nspecies ? ctx->ms[s] : 0.0;
  }
  h.dt = ctx->dt;
  h.E0 = ctx->E0;
  h.np = ctx->np;
  h.steps_done = ctx->steps_done;
  return h;
}

// the mesh sections: device pointer and byte count, in image order from PHI
struct MeshSec {
  void *dev;
  uint64_t bytes;
};

void mesh_sections(pic_ctx *ctx, MeshSec out[7]) {
  const uint64_t g = ctx->g.Ng;
  out[0] = {ctx->phi_h, 16 * g};
  out[1] = {ctx->psi_h, 16 * g};
  out[2] = {ctx->rho_h, 16 * g};
  out[3] = {ctx->A_h, 48 * g};
  out[4] = {ctx->U_h, 48 * g};
  out[5] = {ctx->A_real, 24 * g};
  out[6] = {ctx->J_acc, 24 * g};
}

// Copies between the context's state and an image buffer laid out as the
// checkpoint image (header bytes untouched); `to_image` selects the
// direction, `kind` host or device memory on the image side.
int image_copy(pic_ctx *ctx, unsigned char *b, bool to_image, bool image_on_device) {
  const int d = ctx->g.dim;
  const uint64_t R = ctx->rsize, n = ctx->np, cap = ctx->cap;
  const Layout L = layout(d, (int)R, ctx->np, ctx->g.Ng);
  const cudaMemcpyKind k = to_image ? (image_on_device ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyDeviceToHost)
                                    : (image_on_device ? cudaMemcpyDeviceToDevice
                                                       : cudaMemcpyHostToDevice);
  auto cp = [&](void *dev, uint64_t off, uint64_t bytes) -> int {
    if (bytes == 0) return PIC_OK;
    if (to_image) CK(cudaMemcpyAsync(b + off, dev, bytes, k, ctx->st));
    else CK(cudaMemcpyAsync(dev, b + off, bytes, k, ctx->st));
    return PIC_OK;
  };
  int e;
  for (int l = 0; l < d; l++) {
    if ((e = cp(ctx->cell + l * cap, L.off[Layout::CELL] + 4 * l * n, 4 * n))) return e;
    if ((e = cp((char *)ctx->off + R * l * cap, L.off[Layout::OFF] + R * l * n, R * n))) return e;
  }
  for (int c = 0; c < 3; c++)
    if ((e = cp((char *)ctx->P + R * c * cap, L.off[Layout::P] + R * c * n, R * n))) return e;
  if ((e = cp(ctx->w, L.off[Layout::W], 8 * n))) return e;
  if ((e = cp(ctx->sp, L.off[Layout::SP], 4 * n))) return e;
  if ((e = cp(ctx->id, L.off[Layout::ID], 8 * n))) return e;
  MeshSec ms[7];
  mesh_sections(ctx, ms);
  for (int q = 0; q < 7; q++)
    if ((e = cp(ms[q].dev, L.off[Layout::PHI + q], ms[q].bytes))) return e;
  return PIC_OK;
}

}  // namespace

// A device-side snapshot of the accepted state in the image layout (no
// header, no checksum, no validation: the library's own data), and its
// restore into the same context with the same particle count; for calls
// that run a step and must put the state back (pic_step_vjp).
uint64_t state_snapshot_bytes(const pic_ctx *ctx) {
  return layout(ctx->g.dim, ctx->rsize, ctx->np, ctx->g.Ng).off[Layout::NSEC];
}

int state_snapshot(pic_ctx *ctx, void *dev) {
  return image_copy(ctx, (unsigned char *)dev, true, true);
}

int state_restore(pic_ctx *ctx, const void *dev, int64_t np, long long steps_done,
                  int sort_every, double E0) {
  if (np != ctx->np) {
    ctx->err = "state_restore: particle count changed";
    return PIC_EARG;
  }
  tangent_free(ctx);
  graphs_clear(ctx);
  int e;
  if ((e = image_copy(ctx, (unsigned char *)const_cast<void *>(dev), false, true))) return e;
  if ((e = particles_refresh_A(ctx))) return e;
  ctx->E0 = E0;
  ctx->steps_done = steps_done;
  ctx->opt.sort_every = sort_every;
  ctx->started = 1;
  return PIC_OK;
}

extern "C" {

int pic_checkpoint_bytes(const pic_ctx *ctx, uint64_t *bytes) {
  if (!ctx || !bytes) return PIC_EARG;
  *bytes = layout(ctx->g.dim, ctx->rsize, ctx->np, ctx->g.Ng).off[Layout::NSEC];
  return PIC_OK;
}

int pic_checkpoint_save(pic_ctx *ctx, void *image, uint64_t bytes) {
  if (!ctx || !image) return PIC_EARG;
  if (!ctx->started) {
    ctx->err = "pic_checkpoint_save before pic_start";
    return PIC_ESTATE;
  }
  TraceRange tr("pic_checkpoint_save");
  const Layout L = layout(ctx->g.dim, ctx->rsize, ctx->np, ctx->g.Ng);
  if (bytes != L.off[Layout::NSEC]) {
    ctx->err = "pic_checkpoint_save: buffer size differs from pic_checkpoint_bytes";
    return PIC_EARG;
  }
  unsigned char *b = (unsigned char *)image;
  std::memset(b, 0, bytes);  // section padding is part of the checksum
  int e;
  if ((e = image_copy(ctx, b, true, false))) return e;
  CK(cudaStreamSynchronize(ctx->st));
  pic_checkpoint_header h = header_of(ctx);
  h.total_bytes = bytes;
  h.checksum = fnv1a64(b + sizeof h, bytes - sizeof h);
  std::memcpy(b, &h, sizeof h);
  return PIC_OK;
}

int pic_checkpoint_inspect(const void *image, uint64_t bytes, pic_checkpoint_header *header,
                           char *why, int why_len) {
  const char *msg = "";
  const bool ok = check_image(image, bytes, header, &msg);
  if (why && why_len > 0) {
    std::strncpy(why, msg, (size_t)why_len - 1);
    why[why_len - 1] = '\0';
  }
  return ok ? PIC_OK : PIC_EARG;
}

int pic_checkpoint_load(pic_ctx *ctx, const void *image, uint64_t bytes) {
  if (!ctx) return PIC_EARG;
  TraceRange tr("pic_checkpoint_load");
  pic_checkpoint_header h;
  const char *why = "";
  if (!check_image(image, bytes, &h, &why)) {
    ctx->err = std::string("pic_checkpoint_load: ") + why;
    return PIC_EARG;
  }
  const pic_checkpoint_header mine = header_of(ctx);
  bool same = h.dim == mine.dim && h.precision == mine.precision &&
              h.nspecies == mine.nspecies;
  for (int l = 0; l < 3; l++)
    same = same && h.n[l] == mine.n[l] && h.L[l] == mine.L[l] && h.x0[l] == mine.x0[l];
  for (int s = 0; s < h.nspecies && same; s++)
    same = h.q[s] == mine.q[s] && h.m[s] == mine.m[s];
  if (!same) {
    ctx->err = "pic_checkpoint_load: the image's mesh, precision or species differ from "
               "this context's";
    return PIC_EARG;
  }
  // from here on a failure leaves no usable state: pic_step refuses until
  // a load, pic_set_state or pic_start succeeds
  ctx->started = 0;
  tangent_free(ctx);
  graphs_clear(ctx);
  int e;
  if ((e = particles_alloc(ctx, h.np))) return e;
  ctx->np = h.np;
  // rows of ignorable dimensions are never read; keep them defined
  const uint64_t R = ctx->rsize, n = h.np, cap = ctx->cap;
  for (int l = h.dim; l < 3 && n > 0; l++) {
    CK(cudaMemsetAsync(ctx->cell + l * cap, 0, 4 * n, ctx->st));
    CK(cudaMemsetAsync((char *)ctx->off + R * l * cap, 0, R * n, ctx->st));
  }
  if ((e = image_copy(ctx, (unsigned char *)const_cast<void *>(image), false, false))) return e;
  if ((e = particles_refresh_A(ctx))) return e;
  if ((e = det_alloc(ctx))) return e;
  CK(cudaStreamSynchronize(ctx->st));
  ctx->E0 = h.E0;
  ctx->steps_done = h.steps_done;
  ctx->opt.sort_every = h.sort_every;
  ctx->have_particles = 1;
  ctx->pending_mech = 0;
  ctx->started = 1;
  return PIC_OK;
}

}  // extern "C"

// Differentiated rollout: the recorded forward run and its reverse-mode
// adjoint (see adjoint.cu for the differentiated map).  No counterpart in
// the paper.
//
// Forward (bd_rollout): the ordinary step kernels run with their rollout log
// switched on: the wall reflections of every move, and for every committed
// correction pass its overlapping pairs and the reflected / capped disks.
// Every `every` steps the positions and directions are checkpointed; the
// loss and its gradient with respect to the final positions are formed on
// the device.  The log grows between segments; a segment that overflows it
// is undone (positions, directions, triangulation) and run again with more
// room.
//
// Reverse (bd_rollout_vjp): segments are taken last to first.  Each is
// replayed from its checkpoint with the frozen log, storing the positions at
// every step start and before every correction pass, then the adjoint is
// carried backwards through the passes and moves of the segment.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "bd_handle.h"

struct BdRollout {
  bool recorded = false;
  int nsteps = 0, every = 0, nseg = 0;
  double target = 0.0, loss = 0.0;
  int64_t step0 = 0;
  int npass = 0, npairs = 0;
  std::vector<int> step_pass;    // [nsteps + 1] first pass of each step
  std::vector<int> pass_begin;   // [npass + 1] first pair of each pass
  // log
  uint8_t *refl = nullptr;
  size_t refl_cap = 0;           // bytes
  uint8_t *pflags = nullptr;
  int *pass_begin_d = nullptr;
  int pass_cap = 0;
  int2 *pairs = nullptr;
  int pair_cap = 0;
  int *step_pass_d = nullptr;
  int step_cap = 0;
  // checkpoints and the triangulation at the start of the running segment
  double2 *ck_pos = nullptr;
  float *ck_th = nullptr;
  int ck_cap = 0;
  int4 *tv_seg = nullptr, *tn_seg = nullptr;
  double2 *lam_T = nullptr;      // dL/dx at the final positions
  double *acc = nullptr;         // [0..3] MSD sums, [4] loss, [5] replay loss, [8..12] gradient
  int loss_kind = BD_LOSS_MSD;
  double *hist = nullptr;        // histogram loss: [0, 32) h(x_0), [32, 64) h, [64, 96) dL/dh
  double *hpart = nullptr;       // [np][32] per-disk partial histograms
  // reverse-pass scratch
  double2 *seg_x = nullptr;
  float *seg_th = nullptr;
  int seg_steps_cap = 0;
  double2 *seg_z = nullptr;
  int seg_pass_cap = 0;
  double2 *lam = nullptr, *mud = nullptr, *rpos = nullptr, *rdisp = nullptr, *jpart = nullptr;
  float4 *rwork = nullptr;
  float *rth = nullptr;
  double *gpart = nullptr;
  int jpart_chunks = 0, gpart_cap = 0;
  bool scratch = false;
};

namespace {

using bdcapi::cuda_fail;

// (re)allocate *p for `count` elements, keeping the first `keep` elements
template <class T>
cudaError_t regrow(T **p, size_t keep, size_t count, cudaStream_t s) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(1, count) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (*p && keep) {
    e = cudaMemcpyAsync(q, *p, keep * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaFree(q);
      return e;
    }
  }
  if (*p) cudaFree(*p);
  *p = (T *)q;
  return cudaSuccess;
}

template <class T>
void release(T **p) {
  if (*p) cudaFree((void *)*p);
  *p = nullptr;
}

void detach_log(bd_handle *h) {
  h->d.log_refl = nullptr;
  h->d.log_pflags = nullptr;
  h->d.log_pairs = nullptr;
  h->d.log_pass_begin = nullptr;
  h->d.log_step_pass = nullptr;
  h->c.log_pairs_cap = 0;
  h->c.log_pass_cap = 0;
}

void attach_log(bd_handle *h, BdRollout *r) {
  h->d.log_refl = r->refl;
  h->d.log_pflags = r->pflags;
  h->d.log_pairs = r->pairs;
  h->d.log_pass_begin = r->pass_begin_d;
  h->d.log_step_pass = r->step_pass_d;
  h->c.log_pairs_cap = r->pair_cap;
  h->c.log_pass_cap = r->pass_cap;
}

// room for `passes` more passes and `pairs` more pairs beyond the used part
cudaError_t reserve_log(bd_handle *h, BdRollout *r, int used_pass, int used_pairs, int64_t passes,
                        int64_t pairs) {
  cudaStream_t s = h->stream;
  const size_t np = (size_t)h->np;
  cudaError_t e = cudaSuccess;
  if (used_pass + passes > r->pass_cap) {
    const int64_t want = std::max<int64_t>(used_pass + passes, 2 * (int64_t)r->pass_cap);
    if (want > (1LL << 30)) return cudaErrorMemoryAllocation;
    e = regrow(&r->pflags, (size_t)used_pass * np, (size_t)want * np, s);
    if (e == cudaSuccess) e = regrow(&r->pass_begin_d, (size_t)used_pass + 1, (size_t)want + 1, s);
    if (e != cudaSuccess) return e;
    r->pass_cap = (int)want;
  }
  if (used_pairs + pairs > r->pair_cap) {
    const int64_t want = std::max<int64_t>(used_pairs + pairs, 2 * (int64_t)r->pair_cap);
    if (want > (1LL << 30)) return cudaErrorMemoryAllocation;
    e = regrow(&r->pairs, (size_t)used_pairs, (size_t)want, s);
    if (e != cudaSuccess) return e;
    r->pair_cap = (int)want;
  }
  return cudaSuccess;
}

void add_stats(bd_step_stats *a, const BdCtl &k) {
  a->steps_done += k.st_steps;
  a->corr_iters += k.st_corr_iters;
  a->overlap_pairs += k.st_overlap_pairs;
  a->flip_rounds += k.st_flip_rounds;
  a->flips += k.st_flips;
  a->repair_flips += k.st_repair_flips;
  a->inverted += k.st_inverted;
  a->max_corr_iters = std::max(a->max_corr_iters, k.st_max_corr_iters);
  a->barriers += k.st_barriers;
  double mo;
  unsigned long long bits = k.st_max_overlap_bits;
  memcpy(&mo, &bits, sizeof(mo));
  a->max_overlap = std::max(a->max_overlap, mo);
  if (k.status) {
    a->rejected = 1;
    a->fail_phase = k.st_fail_phase;
    a->fail_item = k.st_fail_item;
    a->fail_count = k.st_fail_count;
  }
}

cudaError_t set_log_cursors(bd_handle *h, int npass, int npairs) {
  int v[4] = {npass, npairs, 0, -1};
  static_assert(offsetof(BdCtl, log_npairs) == offsetof(BdCtl, log_npass) + sizeof(int), "layout");
  static_assert(offsetof(BdCtl, log_step) == offsetof(BdCtl, log_npass) + 3 * sizeof(int), "layout");
  cudaError_t e = cudaMemcpyAsync(&h->d.ctl->log_npass, v, sizeof(v), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e;
}

cudaError_t upload_rep(bd_handle *h) {
  cudaError_t e = cudaMemcpyAsync((void *)h->d.rep, h->h_rep.data(), h->h_rep.size() * sizeof(BdRep),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e;
}

cudaError_t ensure_scratch(bd_handle *h, BdRollout *r) {
  cudaStream_t s = h->stream;
  const size_t np = (size_t)h->np;
  cudaError_t e = cudaSuccess;
  if (!r->scratch) {
    if (e == cudaSuccess) e = regrow(&r->lam, 0, np, s);
    if (e == cudaSuccess) e = regrow(&r->mud, 0, np, s);
    if (e == cudaSuccess) e = regrow(&r->rpos, 0, np, s);
    if (e == cudaSuccess) e = regrow(&r->rdisp, 0, np, s);
    if (e == cudaSuccess) e = regrow(&r->rwork, 0, np, s);
    if (e == cudaSuccess) e = regrow(&r->rth, 0, np, s);
    int jchunk = 0;
    const int nch = bd_adj_force_chunks(h->c, &jchunk);
    const int nbi = (h->np + BD_ADJ_T - 1) / BD_ADJ_T;
    if (e == cudaSuccess) e = regrow(&r->jpart, 0, (size_t)nch * np, s);
    if (e == cudaSuccess) e = regrow(&r->gpart, 0, (size_t)nch * nbi * 5, s);
    if (e != cudaSuccess) return e;
    r->jpart_chunks = nch;
    r->scratch = true;
  }
  if (r->every > r->seg_steps_cap) {
    e = regrow(&r->seg_x, 0, (size_t)r->every * np, s);
    if (e == cudaSuccess) e = regrow(&r->seg_th, 0, (size_t)r->every * np, s);
    if (e != cudaSuccess) return e;
    r->seg_steps_cap = r->every;
  }
  int maxp = 1;
  for (int g = 0; g < r->nseg; ++g) {
    const int t0 = g * r->every, t1 = std::min(r->nsteps, t0 + r->every);
    maxp = std::max(maxp, r->step_pass[t1] - r->step_pass[t0]);
  }
  if (maxp > r->seg_pass_cap) {
    e = regrow(&r->seg_z, 0, (size_t)maxp * np, s);
    if (e != cudaSuccess) return e;
    r->seg_pass_cap = maxp;
  }
  return e == cudaSuccess ? cudaMemsetAsync(r->rdisp, 0, np * sizeof(double2), s) : e;
}

// replay device table: the handle's arrays with the replay's own positions
BdDev replay_dev(const bd_handle *h, const BdRollout *r) {
  BdDev dr = h->d;
  dr.pos = r->rpos;
  dr.work = r->rwork;
  dr.theta = r->rth;
  dr.disp = r->rdisp;
  dr.log_refl = r->refl;
  dr.log_pflags = r->pflags;
  dr.log_pairs = r->pairs;
  dr.log_pass_begin = r->pass_begin_d;
  dr.log_step_pass = r->step_pass_d;
  return dr;
}

// replay steps [t0, t1) from the replay positions; if seg_x is given, store
// the positions and directions at each step start and before each pass
cudaError_t replay(bd_handle *h, BdRollout *r, const BdDev &dr, int t0, int t1, bool store) {
  cudaStream_t s = h->stream;
  const size_t np = (size_t)h->np;
  const int pb0 = r->step_pass[t0];
  cudaError_t e = cudaSuccess;
  for (int t = t0; t < t1 && e == cudaSuccess; ++t) {
    if (store) {
      e = cudaMemcpyAsync(r->seg_x + (size_t)(t - t0) * np, dr.pos, np * sizeof(double2),
                          cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->seg_th + (size_t)(t - t0) * np, dr.theta, np * sizeof(float),
                            cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) e = bd_launch_force_long(dr, h->c, s);
    if (e == cudaSuccess) e = bd_adj_rp_em(dr, h->c, (long long)(r->step0 + t), t, s);
    for (int p = r->step_pass[t]; p < r->step_pass[t + 1] && e == cudaSuccess; ++p) {
      if (store)
        e = cudaMemcpyAsync(r->seg_z + (size_t)(p - pb0) * np, dr.pos, np * sizeof(double2),
                            cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = bd_adj_rp_pass(dr, h->c, p, r->pass_begin[p], r->pass_begin[p + 1], s);
    }
  }
  return e;
}

cudaError_t load_checkpoint(bd_handle *h, BdRollout *r, const BdDev &dr, int g) {
  cudaStream_t s = h->stream;
  const size_t np = (size_t)h->np;
  cudaError_t e = cudaMemcpyAsync(dr.pos, r->ck_pos + (size_t)g * np, np * sizeof(double2),
                                  cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dr.theta, r->ck_th + (size_t)g * np, np * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = bd_launch_work_copy(dr, h->c, s);
  return e;
}

}  // namespace

namespace bdcapi {

void rollout_release(bd_handle *h) {
  BdRollout *r = h ? h->ro : nullptr;
  if (!r) return;
  release(&r->refl);
  release(&r->pflags);
  release(&r->pass_begin_d);
  release(&r->pairs);
  release(&r->step_pass_d);
  release(&r->ck_pos);
  release(&r->ck_th);
  release(&r->tv_seg);
  release(&r->tn_seg);
  release(&r->lam_T);
  release(&r->acc);
  release(&r->hist);
  release(&r->hpart);
  release(&r->seg_x);
  release(&r->seg_th);
  release(&r->seg_z);
  release(&r->lam);
  release(&r->mud);
  release(&r->rpos);
  release(&r->rdisp);
  release(&r->jpart);
  release(&r->rwork);
  release(&r->rth);
  release(&r->gpart);
  delete r;
  h->ro = nullptr;
  detach_log(h);
}

}  // namespace bdcapi

extern "C" {

int bd_set_step(bd_handle *h, int64_t step) {
  if (!h || step < 0) return BD_ERR_ARG;
  h->step = step;
  const long long v = step;
  cudaError_t e = cudaMemcpyAsync(&h->d.ctl->step_dev, &v, sizeof(v), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? BD_OK : cuda_fail(e);
}

int bd_set_force_params(bd_handle *h, const double *alpha, double v0) {
  if (!h) return BD_ERR_ARG;
  if (alpha) {
    for (int k = 0; k < 4; ++k)
      if (!isfinite(alpha[k])) return BD_ERR_ARG;
    for (const RepHost &RH : h->reps)
      if (RH.p.n_species > 2) return BD_ERR_UNSUPPORTED;   // the 4-entry table is 2 x 2
  }
  for (size_t r = 0; r < h->reps.size(); ++r) {
    bd_params &p = h->reps[r].p;
    BdRep &B = h->h_rep[r];
    if (alpha) {
      for (int k = 0; k < 4; ++k) p.alpha[k] = alpha[k];
      bdcapi::rep_set_alpha(B, p.alpha, p.n_species);
    }
    if (isfinite(v0)) {
      p.v0 = v0;
      B.v0 = v0;
    }
  }
  if (h->ro) h->ro->recorded = false;
  cudaError_t e = upload_rep(h);
  return e == cudaSuccess ? BD_OK : cuda_fail(e);
}

int bd_rollout(bd_handle *h, int32_t nsteps, int32_t ckpt_every, int32_t loss_kind, double target,
               double *loss, bd_step_stats *stats) {
  if (!h || nsteps < 1 || ckpt_every < 1 || !isfinite(target)) return BD_ERR_ARG;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (loss_kind != BD_LOSS_MSD && loss_kind != BD_LOSS_HIST) return BD_ERR_UNSUPPORTED;
  if (h->reps.size() != 1 || h->reps[0].p.law != BD_LAW_LONG || h->reps[0].periodic ||
      h->reps[0].p.n_species > 2 || h->d.rad)
    return BD_ERR_UNSUPPORTED;
  if (!h->ro) {
    h->ro = new (std::nothrow) BdRollout;
    if (!h->ro) return BD_ERR_NOMEM;
  }
  BdRollout *r = h->ro;
  r->recorded = false;
  cudaStream_t s = h->stream;
  const size_t np = (size_t)h->np;
  r->nsteps = nsteps;
  r->every = std::min(ckpt_every, nsteps);
  r->nseg = (nsteps + r->every - 1) / r->every;
  r->target = target;
  r->loss_kind = loss_kind;
  r->step0 = h->step;
  cudaError_t e = cudaSuccess;
  if ((size_t)nsteps * np > r->refl_cap) {
    e = regrow(&r->refl, 0, (size_t)nsteps * np, s);
    if (e != cudaSuccess) return cuda_fail(e);
    r->refl_cap = (size_t)nsteps * np;
  }
  if (nsteps + 1 > r->step_cap) {
    e = regrow(&r->step_pass_d, 0, (size_t)nsteps + 1, s);
    if (e != cudaSuccess) return cuda_fail(e);
    r->step_cap = nsteps + 1;
  }
  if (r->nseg > r->ck_cap) {
    e = regrow(&r->ck_pos, 0, (size_t)r->nseg * np, s);
    if (e == cudaSuccess) e = regrow(&r->ck_th, 0, (size_t)r->nseg * np, s);
    if (e != cudaSuccess) return cuda_fail(e);
    r->ck_cap = r->nseg;
  }
  if (!r->tv_seg) {
    e = regrow(&r->tv_seg, 0, (size_t)h->nt, s);
    if (e == cudaSuccess) e = regrow(&r->tn_seg, 0, (size_t)h->nt, s);
    if (e == cudaSuccess) e = regrow(&r->lam_T, 0, np, s);
    if (e == cudaSuccess) e = regrow(&r->acc, 0, 16, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (loss_kind == BD_LOSS_HIST && !r->hist) {
    e = regrow(&r->hist, 0, 96, s);
    if (e == cudaSuccess) e = regrow(&r->hpart, 0, 32 * np, s);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  // log capacity guesses, raised as the rollout shows what it needs
  int64_t pass_per_step = 4, pairs_per_step = std::max<int64_t>(64, h->n / 16);
  int used_pass = 0, used_pairs = 0;
  e = cudaMemsetAsync(r->step_pass_d, 0, sizeof(int), s);
  if (e == cudaSuccess) e = set_log_cursors(h, 0, 0);
  if (e != cudaSuccess) return cuda_fail(e);
  bd_step_stats acc_stats;
  memset(&acc_stats, 0, sizeof(acc_stats));
  int64_t launches = 0;
  for (int g = 0; g < r->nseg; ++g) {
    const int t0 = g * r->every, t1 = std::min(nsteps, t0 + r->every), k = t1 - t0;
    e = cudaMemcpyAsync(r->ck_pos + (size_t)g * np, h->d.pos, np * sizeof(double2), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->ck_th + (size_t)g * np, h->d.theta, np * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->tv_seg, h->d.tv, (size_t)h->nt * sizeof(int4), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r->tn_seg, h->d.tn, (size_t)h->nt * sizeof(int4), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) break;
    for (int attempt = 0;; ++attempt) {
      e = reserve_log(h, r, used_pass, used_pairs, 2 * k * pass_per_step + 16, 2 * k * pairs_per_step + 1024);
      if (e != cudaSuccess) break;
      attach_log(h, r);
      e = bdcapi::reset_stats(h);
      for (int t = t0; t < t1 && e == cudaSuccess; ++t) {
        e = bd_launch_force_long(h->d, h->c, s);
        if (e == cudaSuccess) e = bd_launch_integrate(h->d, h->c, r->step0 + t, t, s);
        if (e == cudaSuccess) e = bd_launch_dt(h->d, h->c, 0, s, h->dt_grid, h->dt_block, t);
        launches += 2 + (h->c.precision == 0 ? bd_force_launches(h->c.force_variant) : 1);
      }
      if (e != cudaSuccess) break;
      int rc = bdcapi::read_ctl(h);
      if (rc) {
        detach_log(h);
        return rc;
      }
      const BdCtl &kc = *h->h_ctl;
      if (kc.status) {
        add_stats(&acc_stats, kc);
        if (stats) *stats = acc_stats;
        detach_log(h);
        h->step = r->step0 + t0;   // the kernels left the state before the failed step
        h->step += kc.st_steps;
        return bdcapi::finish_status(h, kc.status);
      }
      if (!kc.log_overflow) {
        add_stats(&acc_stats, kc);
        bdcapi::add_stage_times(h);
        const int seg_pass = kc.log_npass - used_pass, seg_pairs = kc.log_npairs - used_pairs;
        pass_per_step = std::max<int64_t>(pass_per_step, (seg_pass + k - 1) / k);
        pairs_per_step = std::max<int64_t>(pairs_per_step, (seg_pairs + k - 1) / k);
        used_pass = kc.log_npass;
        used_pairs = kc.log_npairs;
        break;
      }
      // the log ran out of room: undo the segment and run it again with more
      if (attempt >= 8) {
        e = cudaErrorMemoryAllocation;
        break;
      }
      pass_per_step *= 4;
      pairs_per_step *= 4;
      e = cudaMemcpyAsync(h->d.pos, r->ck_pos + (size_t)g * np, np * sizeof(double2), cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d.theta, r->ck_th + (size_t)g * np, np * sizeof(float), cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d.tv, r->tv_seg, (size_t)h->nt * sizeof(int4), cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d.tn, r->tn_seg, (size_t)h->nt * sizeof(int4), cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = bd_launch_work_copy(h->d, h->c, s);
      if (e == cudaSuccess) e = set_log_cursors(h, used_pass, used_pairs);
      if (e == cudaSuccess) {
        // the undone steps had advanced the device step counter
        const long long s0 = r->step0 + t0;
        e = cudaMemcpyAsync(&h->d.ctl->step_dev, &s0, sizeof(s0), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      }
      if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) break;
    h->step = r->step0 + t1;
  }
  detach_log(h);
  h->last_launches = launches;
  if (stats) *stats = acc_stats;
  if (e != cudaSuccess) return cuda_fail(e);
  // loss and dL/dx_T
  if (loss_kind == BD_LOSS_HIST) {
    // the histogram of the start (the first checkpoint), then of x_T against it
    e = bd_adj_hist(h->d, h->c, h->n, r->ck_pos, r->hpart, r->hist, nullptr, nullptr, nullptr, nullptr, 1.0, s);
    if (e == cudaSuccess)
      e = bd_adj_hist(h->d, h->c, h->n, h->d.pos, r->hpart, r->hist + 32, r->hist, r->hist + 64, r->acc + 4,
                      r->lam_T, 1.0, s);
  } else {
    e = bd_adj_msd(h->d, h->c, r->ck_pos, r->acc, target, 1.0, r->lam_T, r->acc + 4, s);
  }
  double lv = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&lv, r->acc + 4, sizeof(double), cudaMemcpyDeviceToHost, s);
  r->step_pass.assign(nsteps + 1, 0);
  r->pass_begin.assign(used_pass + 1, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->step_pass.data(), r->step_pass_d, (nsteps + 1) * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && used_pass > 0)
    e = cudaMemcpyAsync(r->pass_begin.data(), r->pass_begin_d, (used_pass + 1) * sizeof(int),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (r->step_pass[nsteps] != used_pass) return BD_ERR_CUDA;
  r->npass = used_pass;
  r->npairs = used_pairs;
  r->loss = lv;
  r->recorded = true;
  if (loss) *loss = lv;
  return BD_OK;
}

int bd_rollout_vjp(bd_handle *h, double *grad) {
  if (!h || !grad) return BD_ERR_ARG;
  BdRollout *r = h->ro;
  if (!r || !r->recorded) return BD_ERR_ARG;
  cudaStream_t s = h->stream;
  const size_t np = (size_t)h->np;
  cudaError_t e = ensure_scratch(h, r);
  if (e != cudaSuccess) return cuda_fail(e);
  const BdDev dr = replay_dev(h, r);
  int64_t launches = 0;
  e = cudaMemsetAsync(r->acc + 8, 0, 5 * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->lam, r->lam_T, np * sizeof(double2), cudaMemcpyDeviceToDevice, s);
  for (int g = r->nseg - 1; g >= 0 && e == cudaSuccess; --g) {
    const int t0 = g * r->every, t1 = std::min(r->nsteps, t0 + r->every);
    const int pb0 = r->step_pass[t0];
    e = load_checkpoint(h, r, dr, g);
    if (e == cudaSuccess) e = replay(h, r, dr, t0, t1, true);
    for (int t = t1 - 1; t >= t0 && e == cudaSuccess; --t) {
      for (int p = r->step_pass[t + 1] - 1; p >= r->step_pass[t] && e == cudaSuccess; --p) {
        e = bd_adj_vjp_pass(dr, h->c, p, r->pass_begin[p], r->pass_begin[p + 1], r->seg_z + (size_t)(p - pb0) * np,
                            r->lam, r->mud, s);
        launches += 3;
      }
      if (e == cudaSuccess)
        e = bd_adj_vjp_em(dr, h->c, t, r->seg_x + (size_t)(t - t0) * np, r->seg_th + (size_t)(t - t0) * np,
                          r->lam, r->jpart, r->gpart, r->acc + 8, s);
      launches += 4;
    }
  }
  double gh[5] = {0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(gh, r->acc + 8, sizeof(gh), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  h->last_launches = launches;
  // a single-species system has one charge product: report its derivative in slot 0
  if (h->reps[0].p.n_species == 1) {
    gh[0] = gh[0] + gh[1] + gh[2] + gh[3];
    gh[1] = gh[2] = gh[3] = 0.0;
  }
  memcpy(grad, gh, sizeof(gh));
  return BD_OK;
}

int bd_rollout_replay(bd_handle *h, const double *alpha, double v0, double *loss) {
  if (!h || !loss) return BD_ERR_ARG;
  BdRollout *r = h->ro;
  if (!r || !r->recorded) return BD_ERR_ARG;
  if (alpha)
    for (int k = 0; k < 4; ++k)
      if (!isfinite(alpha[k])) return BD_ERR_ARG;
  cudaStream_t s = h->stream;
  cudaError_t e = ensure_scratch(h, r);
  if (e != cudaSuccess) return cuda_fail(e);
  const BdRep saved = h->h_rep[0];
  BdRep &B = h->h_rep[0];
  if (alpha) bdcapi::rep_set_alpha(B, alpha, h->reps[0].p.n_species);
  if (isfinite(v0)) B.v0 = v0;
  e = upload_rep(h);
  const BdDev dr = replay_dev(h, r);
  if (e == cudaSuccess) e = load_checkpoint(h, r, dr, 0);
  if (e == cudaSuccess) e = replay(h, r, dr, 0, r->nsteps, false);
  if (e == cudaSuccess) {
    if (r->loss_kind == BD_LOSS_HIST)
      e = bd_adj_hist(dr, h->c, h->n, dr.pos, r->hpart, r->hist + 32, r->hist, r->hist + 64, r->acc + 5, nullptr,
                      1.0, s);
    else
      e = bd_adj_msd(dr, h->c, r->ck_pos, r->acc, r->target, 1.0, nullptr, r->acc + 5, s);
  }
  double lv = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&lv, r->acc + 5, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  h->h_rep[0] = saved;
  cudaError_t e2 = upload_rep(h);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e);
  *loss = lv;
  return BD_OK;
}

int bd_rollout_positions(bd_handle *h, int32_t which, double *xy) {
  if (!h || !xy || which < 0 || which > 1) return BD_ERR_ARG;
  BdRollout *r = h->ro;
  if (!r || !r->recorded) return BD_ERR_ARG;
  if (which == 1 && !r->scratch) return BD_ERR_ARG;
  const size_t np = (size_t)h->np;
  std::vector<double2> v(np);
  cudaError_t e = cudaMemcpyAsync(v.data(), which == 0 ? (const double2 *)r->ck_pos : (const double2 *)r->rpos,
                                  np * sizeof(double2), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  for (int i = 0; i < h->n; ++i) {
    const double2 p = v[h->int_of_ext[i]];
    xy[2 * i] = p.x;
    xy[2 * i + 1] = p.y;
  }
  return BD_OK;
}

int bd_rollout_log_size(bd_handle *h, int32_t *n_pass, int32_t *n_pairs) {
  if (!h) return BD_ERR_ARG;
  BdRollout *r = h->ro;
  if (!r || !r->recorded) return BD_ERR_ARG;
  if (n_pass) *n_pass = r->npass;
  if (n_pairs) *n_pairs = r->npairs;
  return BD_OK;
}

}  // extern "C"

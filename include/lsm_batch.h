/*
 * lsm_batch.h -- C ABI of the batched 2D lattice-spring path (liblsm.so).
 *
 * Many image-derived specimens of uneven size are stepped together: every
 * time step is one launch of a tile kernel over the tiles of all specimens
 * (the same per-tile step as the single-specimen 2D kernel: spring force,
 * Eq. 2; break test, Section 2.3 force listing; damped velocity Verlet,
 * Eqs. 3-5), the step loop is a cached CUDA graph, and the tile height, grid
 * size and tile order are picked by a built-in autotuner. The paper runs one
 * specimen per program (Section 3.2); batching is this library's addition.
 *
 * Conventions are those of lsm.h (status codes, host buffers owned by the
 * caller, component-major particle arrays, canonical spring order, work
 * ordered on the stream of descs[0]). Specimens are indexed 0..count-1 in
 * input order. All specimens share the material tables, dt, damping, grip
 * and load modes and precision of descs[0]; only the images differ.
 */
#ifndef LSM_BATCH_H
#define LSM_BATCH_H

#include "lsm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsm_batch lsm_batch;

/* Build count 2D specimens (descs[i].dim must be 2). Inputs are copied.
 * Errors: LSM_EINVAL (bad or inconsistent descriptors), LSM_ENOMEM, LSM_ECUDA. */
lsm_status lsm_build_batch(const lsm_desc *descs, int32_t count, lsm_batch **out);

void lsm_batch_destroy(lsm_batch *b);

/* One-line reason for the last failure on b (b == NULL: last build error of
 * the calling thread). */
const char *lsm_batch_last_error(const lsm_batch *b);

/* Number of specimens; particles and springs of specimen spec (outputs may be
 * NULL). */
lsm_status lsm_batch_sizes(lsm_batch *b, int32_t spec, int32_t *count, int64_t *n, int64_t *m);

/* Time steps_per_trial steps of every candidate schedule (tile height
 * 8/16/32, grid of one CTA per tile or a persistent grid of 4 or 8 CTAs per
 * SM, natural or largest-specimen-first tile order; in the F32 and DF modes
 * also the strip schedules -8/-16/-32, below) on a copy of the current
 * state, after a warm-up that brings the GPU to its load clocks, in two
 * sweeps; keep the schedule with the fastest trial and restore the state.
 * Outputs (may be NULL): chosen tile height (negative: strips of that many
 * rows), grid size (0 = one CTA per tile), order (0 natural, 1 largest
 * first) and its time per step in ms. */
lsm_status lsm_batch_autotune(lsm_batch *b, int32_t steps_per_trial, int32_t *tile_y, int32_t *grid,
                              int32_t *order, double *ms_per_step);

/* Set the schedule explicitly: tile_y 8, 16 or 32 (tiles of 32 columns and
 * that many rows, one CTA each), or -8, -16, -32 (F32 and DF modes, every
 * specimen below 2^29 pixels): the time steps run as one warp per strip of
 * 30 owned columns and 8, 16 or 32 rows, the register-resident sweep of the
 * single-specimen strip kernel (sample sums per strip), while load
 * increments keep 16-row tiles; the states are the same bits either way.
 * grid >= 0 (tiles only); order 0 or 1. LSM_EINVAL otherwise. A new batch
 * starts with strips of 16 rows (F32, DF, when they outnumber the warps the
 * device holds at once) or 16-row tiles, largest specimens first, grid 0. */
lsm_status lsm_batch_set_schedule(lsm_batch *b, int32_t tile_y, int32_t grid, int32_t order);

/* Load increment of every specimen to the absolute strains eps[0..count-1]
 * (host array), as lsm_apply_strain does for one specimen. */
lsm_status lsm_batch_apply_strain(lsm_batch *b, const double *eps);

/* nsteps time steps of every specimen (force Eq. 2, break test, damped
 * velocity Verlet Eqs. 3-5, as lsm_step), then one sample per specimen.
 * Stream-ordered (a cached CUDA graph per nsteps). */
lsm_status lsm_batch_step(lsm_batch *b, int64_t nsteps);

/* Relax every specimen to a force residual (the quasi-static limit of the
 * damped dynamics, Section 2.2): steps in batches of check_every;
 * after each batch every specimen whose residual is <= tol stops stepping.
 * Returns when all have converged or after max_steps steps. taken[i] (host,
 * may be NULL) = steps specimen i ran; converged[i] = 1 if it met tol. One
 * sample per specimen is recorded at the end. Returns LSM_OK, or LSM_ENOTCONV
 * if any specimen did not converge. Synchronises after every batch. */
lsm_status lsm_batch_relax(lsm_batch *b, double tol, int64_t max_steps, int64_t check_every,
                           int64_t *taken, int32_t *converged);

/* Recorded samples of specimen spec (see lsm_samples). Synchronises. */
lsm_status lsm_batch_samples(lsm_batch *b, int32_t spec, lsm_sample *out, int64_t cap, int64_t *count);

/* State of specimen spec (dim*n doubles each, component-major; either may be
 * NULL). Synchronises. */
lsm_status lsm_batch_get_state(lsm_batch *b, int32_t spec, double *x, double *v);

/* Replace the positions and/or velocities of specimen spec; its acceleration
 * is re-evaluated (Eq. 4). Synchronises. */
lsm_status lsm_batch_set_state(lsm_batch *b, int32_t spec, const double *x, const double *v);

/* Broken-spring mask of specimen spec in canonical order (cap >= its m) and
 * the index of its first step with a break (-1 if none). Synchronises. */
lsm_status lsm_batch_broken_mask(lsm_batch *b, int32_t spec, uint8_t *out, int64_t cap, int64_t *m,
                                 int64_t *first_break_step);

/* Spring updates evaluated (sum over specimens of springs x steps taken) and
 * kernels launched by the library so far. */
lsm_status lsm_batch_counters(lsm_batch *b, int64_t *spring_updates, int64_t *kernel_launches);

/* Wait for queued work; returns any pending device status. */
lsm_status lsm_batch_synchronize(lsm_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* LSM_BATCH_H */

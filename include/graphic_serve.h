/*
 * graphic_serve.h -- serving loop of the GRAPHIC GB300 library: full ADI
 * reductions (Sect. 3: recentring shift, angle-gated median PSF subtraction,
 * derotation, median collapse -- the arithmetic of graphic_reduce) requested
 * by many clients, for cubes of different sizes, run with continuous
 * cross-request batching on one GPU.
 *
 * Model.  A native scheduler thread owns a device arena (the admission
 * budget) and two library contexts.  Requests are admitted first come first
 * served as soon as their cube, result and plan fit in the arena and fewer
 * than max_active requests are resident; the cube is copied in on a copy
 * stream while other requests compute.  Work advances in iterations: each
 * iteration moves every resident request one stage on (shift -> median PSF
 * subtraction -> derotation -> collapse and copy-out); the shift and
 * derotation stages of all requests in an iteration run as ONE uneven batch
 * (graphic_batch_geom, the configured mode), the median stages as one launch
 * per request.  Up to two iterations are in flight, so requests that arrive
 * while others are on the GPU join the next iteration.  Every request's
 * result is independent of what it was batched with (the same kernels, the
 * same per-frame arithmetic): with the grouped or per-cube batch modes
 * bit-identical to graphic_reduce under the same schedule, with the
 * persistent mode (generic kernel for 1024-point lines) within 1e-5 of the
 * cube's peak.
 *
 * Host memory.  host_in must stay valid and unchanged until the request
 * completes; pinned memory (cudaHostAlloc, torch pin_memory) makes its copy
 * asynchronous, pageable memory stalls the scheduler for the copy.  The
 * result is written to host_out before graphic_server_wait reports the
 * request done.  Per-frame arrays are copied at submit.
 *
 * Errors: the GRAPHIC_ERR_* codes of graphic.h; a request whose cube can
 * never fit in the budget fails with GRAPHIC_ERR_OOM, a non-finite input
 * with GRAPHIC_ERR_NONFINITE (in that request only).
 */
#ifndef GRAPHIC_SERVE_H
#define GRAPHIC_SERVE_H

#include <stdint.h>

#include "graphic.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct graphic_server graphic_server;

typedef struct {
  int32_t device;
  int32_t max_active;        /* requests resident on the device at once (0: 16)                        */
  int32_t batch_mode;        /* geometric stages: GRAPHIC_BATCH_* (GRAPHIC_BATCH_AUTO: the schedule's)  */
  int32_t reserved;          /* 0                                                                      */
  int64_t max_device_bytes;  /* admission budget (0: 150 GiB); capped by free HBM minus workspaces     */
  int64_t staging_bytes;     /* pinned host staging for plans and results (0: 256 MiB)                 */
} graphic_server_config;

/* One reduction: the arguments of graphic_reduce with host buffers. */
typedef struct {
  const float *host_in;      /* n_frames x n x n                                   */
  float *host_out;           /* n x n median-collapsed residual                    */
  int64_t n_frames;
  int32_t n;
  int32_t n_edges;           /* annulus edges (>= 2)                               */
  const double *dx;          /* [n_frames] recentring shifts (Sect. 3.3.1)         */
  const double *dy;
  const double *parang;      /* [n_frames] parallactic angles, degrees (Sect. 3.3) */
  const double *edges;       /* [n_edges] annulus radii, px, increasing            */
  double fwhm;
  double n_fwhm;
} graphic_request;

typedef struct {
  int32_t status;            /* GRAPHIC_OK or the request's error code             */
  int32_t reserved;
  double t_submit;           /* seconds on the server clock (graphic_server_clock) */
  double t_admit;            /* device memory granted, copy-in enqueued            */
  double t_done;             /* result in host_out                                 */
} graphic_request_info;

typedef struct {
  int64_t submitted, admitted, completed, failed;
  int64_t iterations;        /* iterations issued                                  */
  int64_t batch_launches;    /* geometric batch calls                              */
  int64_t batch_items;       /* request stages in them (items / launches: mean batch) */
  int64_t max_batch_items;
  int64_t max_resident;      /* most requests resident at once                     */
  int64_t device_bytes_cap;  /* arena size                                         */
  int64_t device_bytes_peak; /* arena high-water mark                              */
} graphic_server_stats;

/* Start a server on cfg->device (cfg may be NULL: defaults).  Allocates the
 * arena and the pinned staging up front. */
int graphic_server_create(graphic_server **out, const graphic_server_config *cfg);

/* Queue one request; *id receives its handle.  Arguments are checked here
 * (as graphic_reduce checks them). */
int graphic_server_submit(graphic_server *s, const graphic_request *r, int64_t *id);

/* Wait up to timeout_s seconds (< 0: no limit) for request `id`; on return
 * with GRAPHIC_OK, info (may be NULL) is filled and the handle is released;
 * info->status is the request's own result code.  GRAPHIC_ERR_TIMEOUT if the
 * request is still running (the handle stays valid). */
int graphic_server_wait(graphic_server *s, int64_t id, double timeout_s, graphic_request_info *info);

/* Seconds since the server started (the clock of graphic_request_info). */
double graphic_server_clock(graphic_server *s);

int graphic_server_stats_read(graphic_server *s, graphic_server_stats *st);

/* Finish every submitted request, stop the scheduler, free everything. */
int graphic_server_destroy(graphic_server *s);

#ifdef __cplusplus
}
#endif

#endif /* GRAPHIC_SERVE_H */

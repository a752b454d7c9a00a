/*
 * piccs_server.h -- request loop for repeated scans (C ABI).
 *
 * The setting of the paper (Sec. 1, Sec. 3): during an image-guided procedure
 * a patient is scanned again and again with the same geometry, each new scan
 * reconstructed against that patient's prior volume.  A server keeps, per
 * patient, a session on the device -- the geometry's ray tables, the prior,
 * and the workspace of up to max_batch scans (a batched piccs context) --
 * and takes reconstruction requests as they arrive:
 *
 *   - admission by HBM footprint: a patient's session is created when a
 *     request for it arrives and its workspace fits in the budget, evicting
 *     the least recently used idle sessions if needed; a request whose
 *     session cannot be made resident yet waits in its queue;
 *   - continuous batching: when a session is idle, the requests queued for
 *     it that share parameters (up to max_batch) are reconstructed together,
 *     one launch per kernel for all of them; requests arriving meanwhile join
 *     the next batch.  Long scans (estimated 200 ms or more) are batched only
 *     while more than 2 * max_batch requests are queued in all: they gain
 *     little from sharing launches, and the first scan of a batch waits for
 *     all of it;
 *   - order: among idle sessions with queued requests, the one whose oldest
 *     request has the highest response ratio (time waited + estimated device
 *     time) / estimated device time goes first, so short scans overtake long
 *     ones while no request waits without bound -- or the oldest request
 *     first, or (adaptive) the former only under a backlog;
 *   - overlap: up to max_running batches (of different patients) are in
 *     flight at once, each on its session's own CUDA stream, as long as each
 *     is small (estimated below 25 ms of device time per scan); a scan that
 *     fills the GPU on its own runs alone, since overlapping it would only
 *     stretch both batches;
 *   - scans of different sizes together: when the session going next has a
 *     short scan (estimated below 200 ms) at the head of its queue, up to
 *     max_group - 1 further idle sessions -- other patients, other
 *     geometries -- whose oldest requests have the same parameters join it,
 *     in issue order, each with its batch: the group runs as one
 *     reconstruction in lockstep, every product with A and with A^T one
 *     kernel launch for all of them (piccs_run_staged_group), and counts as
 *     one batch in flight;
 *   - captured launches: for scans estimated below 200 ms (where launch
 *     costs matter), a session records the launch sequence of each
 *     (parameters, batch size) pair once as a CUDA graph and replays it;
 *     a group's sequence is one graph per (sessions, batch sizes, parameters).
 *
 * All calls are thread-safe.  A worker thread owned by the server issues
 * every CUDA call for the sessions on the device that was current when the
 * server was created.  Results are bit-identical to piccs_reconstruct of the
 * same scan alone (the batched kernels are the single-scan kernels per slot).
 */
#ifndef PICCS_SERVER_H
#define PICCS_SERVER_H

#include <stddef.h>

#include "piccs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct piccs_server piccs_server;

typedef struct {
    size_t hbm_budget;  /* device bytes the sessions may hold (0: 90% of the
                           memory free when the server is created) */
    int max_batch;      /* scans of one patient reconstructed together (1..64) */
    int max_running;    /* batches in flight at once (>= 1) */
    int use_graphs;     /* replay captured CUDA graphs for short scans (0: never) */
    int order;          /* PICCS_ORDER_*: which idle session's queue goes next */
    int max_group;      /* sessions of different patients run as one group
                           (0 or 1: never; at most 8) -- see above */
} piccs_server_config;

/* Issue order among idle sessions with queued requests: by the highest
 * response ratio (time waited + estimated device time) / estimated device
 * time of their oldest request (short scans overtake long ones; favours the
 * median latency), first come first served (the oldest request first), or
 * adaptive: response ratio while more than 2 * max_batch requests are
 * queued (a backlog worth reordering), first come first served otherwise
 * (with a short queue, reordering only makes the overtaken scan wait). */
enum { PICCS_ORDER_RESPONSE_RATIO = 0, PICCS_ORDER_FIFO = 1, PICCS_ORDER_ADAPTIVE = 2 };

typedef struct {
    int status;          /* PICCS_OK or the request's error (PICCS_E*) */
    int batch;           /* scans in the batch the request ran in */
    double queued_ms;    /* submission -> its batch was issued */
    double run_ms;       /* issued -> result on the host */
    double total_ms;     /* submission -> result on the host */
} piccs_request_stats;

typedef struct {
    long long submitted, completed, failed;
    long long batches;         /* batches issued */
    long long graph_replays;   /* batches issued as one graph launch */
    long long sessions_made;   /* sessions created (including re-creations) */
    long long evictions;       /* sessions evicted to admit others */
    size_t hbm_in_use;         /* bytes held by resident sessions */
    long long group_runs;      /* issues that ran several sessions as one group */
} piccs_server_stats;

/* Start a server (and its worker thread).  PICCS_EINVAL on a bad config. */
int piccs_server_create(piccs_server **out, const piccs_server_config *cfg);

/* Finish every queued request, stop the worker, free all sessions. */
void piccs_server_destroy(piccs_server *srv);

/* Message of the last failing call on srv (NULL srv: of piccs_server_create
 * on this thread); valid until this thread's next call of this function. */
const char *piccs_server_last_error(const piccs_server *srv);

/* Register patient `patient` (any int not yet registered): its geometry and
 * prior volume (M floats, host; copied) are kept on the host until a request
 * makes the session resident.  PICCS_EINVAL on a bad geometry, PICCS_ENOMEM
 * if its session alone exceeds the budget. */
int piccs_server_add_patient(piccs_server *srv, int patient, const piccs_geometry *geometry,
                             const float *h_xprior);

/* Queue a reconstruction of patient `patient` (x0_mode PRIOR or ZERO).
 * h_proj holds N projection values: FP32, or BF16 bit patterns when
 * params->storage is PICCS_STORAGE_BF16 (half the bytes to move).
 * h_proj is read and h_out (M floats) written asynchronously, so
 * both must stay valid, and h_proj unchanged, until piccs_server_wait reports
 * the request done; pinned host memory lets the copies overlap.  Returns at
 * once with the request's ticket. */
int piccs_server_submit(piccs_server *srv, int patient, const void *h_proj,
                        const piccs_params *params, float *h_out, long long *ticket);

/* Wait for a request (timeout_ms < 0: without limit).  PICCS_ETIMEOUT if it
 * is still pending when the time is up; else PICCS_OK with *st filled (the
 * request's own status in st->status).  A ticket can be waited for once. */
int piccs_server_wait(piccs_server *srv, long long ticket, int timeout_ms,
                      piccs_request_stats *st);

/* Counters since creation. */
int piccs_server_get_stats(piccs_server *srv, piccs_server_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* PICCS_SERVER_H */

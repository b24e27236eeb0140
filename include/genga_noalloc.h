/*
 * genga_noalloc.h -- a long-range kick that allocates no device memory.
 *
 * The paper has no counterpart for this entry point.  It exists for callers
 * that cannot call cudaMalloc: code running inside another framework's
 * memory pool or allocator hooks, plug-ins that may not grow device memory,
 * and hosts that fix their device-memory budget up front.  genga_kick needs
 * a context whose workspace genga_create allocates; this entry point needs
 * none.
 */
#ifndef GENGA_NOALLOC_H
#define GENGA_NOALLOC_H

#include "genga.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest N genga_kick_noalloc accepts.  Its scratch is a fixed __device__
 * array of 3 * GENGA_NOALLOC_MAX_N + 256 doubles (about 1.6 MB) that every
 * GPU which loads the library keeps until the process exits. */
#define GENGA_NOALLOC_MAX_N 65536

/*
 * The FP64 long-range kick of genga_kick (same sum, critical radius and
 * changeover weight, same acc layout acc[c*N + i] and v += acc * tau), run on
 * the CURRENT device without allocating device memory.  The caller owns
 * `sys`'s arrays and `acc` (device, or NULL to skip it); the kernels' scratch
 * lives in a static device array shared by every call.
 *   params->precision must be GENGA_FP64.
 *   N > GENGA_NOALLOC_MAX_N, bad pointers or parameters: GENGA_ERR_INVALID_ARG,
 *   nothing is enqueued.
 * The first call in each CUDA context (the current device's primary context,
 * or whichever context the caller has made current) looks up the scratch
 * array's device address there (cudaGetSymbolAddress) and keeps it for that
 * context only; a new context -- after cudaDeviceReset, say -- gets its own
 * lookup on its first call.  Make that first call before any stream capture.
 * The scratch keeps the last call's contents and
 * is re-initialised by each call; calls that overlap on the GPU (several
 * streams or host threads at once) race on it and must be serialised by the
 * caller.  No encounter list and no sticky status are produced.
 */
genga_status genga_kick_noalloc(const genga_system *sys, const genga_params *params, double tau, double *acc,
                                void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GENGA_NOALLOC_H */

/*
 * soax_host.h -- particles held in host memory, streamed through the device.
 *
 * The calls of soax.h work on particles resident in device planes, as the paper's GPU
 * container does (Sec. 4.2.2: host-device transfers are costly, so the data should live
 * on the device and cross to the host only when the host needs it).  This header adds
 * one call for a particle set whose home is host memory: one sort interval (the fused
 * steps with the cell keys, the stable cell sort, the permute-gather of every array as
 * in Listing 7's apply) with the set uploaded before and downloaded after, in pieces,
 * so that the copies in the two directions and the steps overlap one another and the
 * transfer cost is paid once per interval at the link's combined rate.  Conventions
 * (return codes, validation, ownership, alignment) are those of soax.h.
 */
#ifndef SOAX_HOST_H
#define SOAX_HOST_H

#include "soax.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One sort interval of the particles in host memory, in nchunks pieces of consecutive
 * particles:
 *   1. piece by piece, the host planes are copied into the live device planes
 *      (up_stream), and each piece is advanced nsteps midpoint-RK2 steps with the cell
 *      keys of its final positions written (soax_step_fused_keys on that piece, stream)
 *      as soon as its copy has landed;
 *   2. the stable radix sort of all the keys (soax_sort_perm, stream);
 *   3. piece by piece, the permute-gather of every plane into the other buffer set
 *      (soax_permute restricted to those outputs, stream) and its copy back into the
 *      host planes (down_stream).
 * On return the work is enqueued.  Once down_stream has passed the call the host planes
 * hold the stepped particles in cell order, bit-identical to soax_step_fused_keys +
 * soax_sort_perm + soax_permute on device-resident planes; once stream has passed it the
 * device planes hold the same (the live set has flipped, as after soax_permute).
 *
 *  host:    nplanes pointers (soax_size), in plane order -- fields in schema order, the
 *           components of a field in order -- each to n elements of the plane's type.
 *           Read on entry, overwritten with the result.  Page-locked (pinned) memory
 *           makes the copies asynchronous and lets them overlap; pageable memory works
 *           but serialises them.  The caller must not touch them until down_stream
 *           has passed the call.
 *  fl, nsteps (>= 0), grid (1..1024): as for soax_step_fused_keys.
 *  nchunks: pieces (0 = 16); at most one piece per 16 particles is used.
 *  defer:   0: the call enqueues its downloads.  1: it leaves them to the next
 *           soax_step_host call on this handle, which enqueues each piece's download just
 *           before its own upload of the same piece and holds it back until its upload
 *           two pieces earlier has landed, so the two link directions move together
 *           instead of the downloads running ahead; or to soax_step_host_finish.  Until
 *           one of those has been enqueued, the live device planes must not be modified
 *           or rebound (they are what will be downloaded), and the host planes of the
 *           deferred call are final only once down_stream has passed it.
 *  ws:      soax_sort_workspace_bytes(h, grid) bytes (16-byte aligned): the keys and the
 *           permutation (soax_sort_results gives the permutation afterwards).
 *  stream, up_stream, down_stream: the steps, sort and gathers run on stream, the copies
 *           to the device on up_stream and back on down_stream; NULL is the legacy
 *           default stream (which serialises everything).  The call starts after the
 *           work already enqueued on stream.  stream does not wait for the downloads (a
 *           following call's uploads overlap them); synchronise down_stream, or make
 *           stream wait for it, before reading the host planes.
 * Consecutive calls on a handle may be enqueued without synchronising: a piece's upload
 * waits for the previous call's download of the same particles.  Not for stream capture:
 * the downloads end on down_stream, which stream does not join, and a call waits on
 * events the previous call recorded.  For this the handle
 * keeps 3 nchunks + 1 CUDA events of the current device, created at the first call and
 * released by soax_destroy.  Both buffer sets must be bound.  Errors: SOAX_EINVAL (NULL
 * host pointer, bad nsteps, grid or nchunks), SOAX_ESCHEMA (flow fields), SOAX_ENOMEM
 * (workspace too small), SOAX_EALIGN, SOAX_EUNBOUND; all before any copy or launch.
 * SOAX_ECUDA if an event, copy or launch cannot be made (work enqueued before it
 * stays enqueued; a deferred call's downloads are then dropped).  Validation also
 * rejects defer other than 0 or 1.
 * Defining passages: host-device transfers and keeping the data on the device (Sec.
 * 4.2.2); Eq. 1 (Sec. 2) for the steps; spatial locality (Sec. 1) for the cell order;
 * apply-to-all-arrays (Listing 7) for the gather. */
int soax_step_host(soax_t h, void* const* host, const soax_flow* fl, int32_t nsteps, int32_t grid, int32_t nchunks,
                   int32_t defer, void* ws, size_t ws_bytes, void* stream, void* up_stream, void* down_stream);

/* Enqueue, on down_stream, the downloads a soax_step_host call with defer = 1 left
 * (nothing if none are pending); the host planes are final once down_stream has passed
 * them.  SOAX_EINVAL for a NULL handle; SOAX_ECUDA if a copy cannot be enqueued (the
 * deferred call's host planes are then undefined). */
int soax_step_host_finish(soax_t h, void* down_stream);

#ifdef __cplusplus
}
#endif

#endif /* SOAX_HOST_H */

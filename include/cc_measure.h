/*
 * cc_measure.h - a measured ceiling for the edge pass's endpoint lookups.
 *
 * Every edge of the hooking pass (Algorithm 3) looks up both endpoints before
 * it can be dropped: under f = R (Eq. 1) with the zero-tree bitmap, one bit
 * of a bitmap of n/8 bytes per endpoint; otherwise the endpoint's entry of the
 * parent array P. These are 4-byte reads at scattered addresses, one L2
 * request each, so the pass can go no faster than the device serves random
 * 4-byte loads from an array of that size. HBM bandwidth is not that limit:
 * 2 lookups per 8-byte edge use one 32-byte sector each.
 *
 * cc_measure_random_loads times that service rate on the current device, so
 * the edge pass can be reported against it beside the HBM roofline.
 */
#ifndef CC_MEASURE_H
#define CC_MEASURE_H

#include <stdint.h>

#include "cc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Rate of random 4-byte loads (loads per second) on the current device.
 *  - In: array_bytes, the size of the array read, a power of two in
 *    [2^16, 2^32]. Arrays that fit L2 (129 MB on GB300) give the L2 request
 *    ceiling; larger ones add DRAM latency and sector traffic.
 *  - Out: *loads_per_second, the best of several launch shapes (4 or 8
 *    independent loads per thread, L1-allocating or L2-only loads), each
 *    timed with CUDA events over 3 launches after a warm-up launch. Every
 *    load reads an address drawn from a per-thread linear congruential
 *    sequence, uniform over the array.
 *  - Resources: allocates the array (cudaMalloc) and a stream, synchronises,
 *    and frees both before it returns. Takes about 20 ms.
 * Errors: CC_ERR_INVALID_ARGUMENT (NULL out pointer, array_bytes not a power
 * of two in range), CC_ERR_OOM, CC_ERR_CUDA. */
CC_API cc_status cc_measure_random_loads(uint64_t array_bytes, double *loads_per_second);

#ifdef __cplusplus
}
#endif

#endif /* CC_MEASURE_H */

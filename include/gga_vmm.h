/*
 * gga_vmm.h -- the memMap comparison array (the paper's Sec. II
 * "Semi-static" array grown with the low-level virtual memory API, the
 * memMap row of Table II): a flat array whose capacity grows without any
 * copy, by mapping more physical memory behind a range of virtual addresses
 * reserved once.  Indexing stays contiguous; the physical memory is not.
 * It is a baseline the GGArray is measured against, not part of the
 * GGArray.  Error codes are gga.h's.
 *
 * The driver's virtual memory entry points are looked up at run time
 * through the CUDA runtime (the library does not link libcuda, so it still
 * loads where no GPU driver is installed); where they cannot be found every
 * call returns GGA_ERR_CUDA.  All calls are host calls that return when the
 * mapping is done (they do not use a stream).
 */
#ifndef GGA_VMM_H
#define GGA_VMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gga_vmm_t* gga_vmm;

/* Reserve max_bytes (rounded up to the allocation granularity) of device
 * virtual addresses for the current device; nothing is mapped yet.
 * out: host pointer receiving the handle. */
int gga_vmm_create(uint64_t max_bytes, gga_vmm* out);

/* Map physical device memory so that at least the first `bytes` of the
 * range are backed (rounded up to the granularity; one new physical
 * allocation for the part not mapped yet).  Never shrinks, never moves or
 * copies what is mapped.  GGA_ERR_TOO_LARGE beyond the reserved range,
 * GGA_ERR_CUDA if the driver refuses (e.g. out of memory: nothing changes). */
int gga_vmm_grow(gga_vmm v, uint64_t bytes);

/* out3 (host, 3 uint64): device address of the range, bytes mapped,
 * allocation granularity. */
int gga_vmm_info(gga_vmm v, uint64_t* out3);

/* Synchronizes the device, unmaps and frees everything. */
int gga_vmm_destroy(gga_vmm v);

#ifdef __cplusplus
}
#endif

#endif  // GGA_VMM_H

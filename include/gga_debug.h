/*
 * gga_debug.h -- test hooks for the failure paths of the GPU code (not
 * part of the GGArray's operations).  Error codes are gga.h's.
 */
#ifndef GGA_DEBUG_H
#define GGA_DEBUG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * gga_debug_wait_timeout -- one block initializes an mbarrier for one
 * arrival and waits for its phase with the same bounded wait the TMA kernels
 * use, giving up after `attempts` tries.  With arrive = 1 a thread arrives
 * first, so the wait completes: GGA_OK.  With arrive = 0 nothing ever
 * arrives, the wait gives up and the kernel records GGA_ERR_TIMEOUT in a
 * status word and returns (no trap, the context stays usable).  Synchronizes
 * `stream` and returns the recorded status (GGA_ERR_CUDA if a CUDA call
 * failed).  attempts must be in [1, 2^20].
 */
int gga_debug_wait_timeout(uint32_t attempts, int arrive, void* stream);

#ifdef __cplusplus
}
#endif

#endif  // GGA_DEBUG_H

/*
 * gga_flat.h -- the parallel insertion approaches of the paper's Sec. III-B,
 * on a static (flat) array, as its insertion experiment measures them
 * (Sec. VI-A: insertion algorithms are independent of the structure, and
 * the flat array isolates their cost).  Not part of the GGArray: the
 * GGArray's own insertion is gga_insert / gga_insert_generated.  Error
 * codes are gga.h's.
 */
#ifndef GGA_FLAT_H
#define GGA_FLAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  GGA_FLAT_ATOMIC = 0,  /* every thread takes its position with one atomicAdd on the size */
  GGA_FLAT_SCAN = 1     /* warp-shuffle prefix sum in the block, one atomicAdd per block */
};

/*
 * gga_flat_insert -- n_threads threads, in blocks of threads_per_block
 * (32..1024, a multiple of 32), each append one uint32 with value
 * first_value + (its thread index) after the array's current size.
 * array: device, `capacity` uint32; size_dev: device uint64, read and
 * advanced by n_threads.  Which position a thread gets depends on the order
 * the atomics are served in, so the array holds the inserted values in no
 * fixed order (one block's run is contiguous and in thread order with
 * GGA_FLAT_SCAN).  A thread whose position is >= capacity writes nothing
 * (the size still advances; the caller compares it with the capacity).
 */
int gga_flat_insert(int mode, uint32_t* array, uint64_t capacity, uint64_t* size_dev, uint64_t n_threads,
                    uint32_t threads_per_block, uint32_t first_value, void* stream);

#ifdef __cplusplus
}
#endif

#endif  // GGA_FLAT_H

// Device error flags of a sieve and the status cs_sync reports for them.
// Kernels OR these bits into the plan's error word instead of trapping; the
// host reads the word after the sieve and maps it to one status, the most
// fundamental first (a lost prime or hit makes the result invalid).
#pragma once
#include <stdint.h>

#include "../../include/combsieve.h"

namespace cs {

enum Err : uint64_t {
    ERR_PRIME_OVERFLOW = 1,   // a prime chunk produced more primes than its buffer holds
    ERR_SOLVER_LIMIT = 2,     // the solver exceeded its pass bound (never expected)
    ERR_STAGE_TIMEOUT = 4,    // a bounded wait for a shared-memory staging copy gave up
};

inline cs_status status_of_device_errors(uint64_t err, const char **msg) {
    if (err & ERR_PRIME_OVERFLOW) {
        *msg = "prime buffer overflow";
        return CS_EOVERFLOW;
    }
    if (err & ERR_SOLVER_LIMIT) {
        *msg = "modular solver exceeded its pass bound";
        return CS_EDEVICE;
    }
    if (err & ERR_STAGE_TIMEOUT) {
        *msg = "tile sieve: a staging copy did not complete";
        return CS_ETIMEOUT;
    }
    if (err) {
        *msg = "unknown device error flag";
        return CS_EDEVICE;
    }
    *msg = "";
    return CS_OK;
}

}  // namespace cs

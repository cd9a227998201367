// Batched solves over many independent meshes (placeholder until the
// persistent batched kernels land).
#include "sem_internal.h"

using namespace sem;

extern "C" {

SEM_API int sem_cg_solve_batch(sem_handle* h, double* x, const double* b, const sem_solve_opts* opts,
                               sem_solve_stats* stats, cudaStream_t s) {
    (void)x; (void)b; (void)opts; (void)stats; (void)s;
    if (!h) return fail(SEM_EINVAL, "null handle");
    return fail(SEM_EINVAL, "batched solve not available in this build");
}

}  // extern "C"

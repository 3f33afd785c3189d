// Batched multi-system / multi-RHS engine and serving loop (in progress).
#include "gbs_impl.cuh"

extern "C" int gbs_ksp_solve_cg_batched(gbs_ctx, int, const gbs_mat *, const gbs_vec *, gbs_vec *,
                                        const int *, const double *, int, int, int *, double *,
                                        int *)
{
    return GBS_ERR_UNSUPPORTED;
}
extern "C" int gbs_server_create(gbs_ctx, size_t, int, int, gbs_server *) { return GBS_ERR_UNSUPPORTED; }
extern "C" int gbs_server_destroy(gbs_server) { return GBS_OK; }
extern "C" int gbs_server_submit(gbs_server, int64_t, const int32_t *, const int32_t *,
                                 const double *, int, const double *, double, int, uint64_t *)
{
    return GBS_ERR_UNSUPPORTED;
}
extern "C" int gbs_server_progress(gbs_server, int *) { return GBS_ERR_UNSUPPORTED; }
extern "C" int gbs_server_poll(gbs_server, uint64_t, int *) { return GBS_ERR_UNSUPPORTED; }
extern "C" int gbs_server_wait(gbs_server, uint64_t) { return GBS_ERR_UNSUPPORTED; }
extern "C" int gbs_server_fetch(gbs_server, uint64_t, double *, int *, double *, int *)
{
    return GBS_ERR_UNSUPPORTED;
}
extern "C" int gbs_server_stats(gbs_server, int *, int *, int *, size_t *) { return GBS_ERR_UNSUPPORTED; }

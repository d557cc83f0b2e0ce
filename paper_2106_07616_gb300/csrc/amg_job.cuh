// amg_job.cuh -- the multigrid hierarchy build of amg.cuh split in two, so
// that its host part runs on a thread of its own while the device works.
#pragma once
#include "amg.cuh"

namespace rbffd {

// The same build in two halves.  amg_build_begin builds level 0 on the
// device first when it applies (amg_setup.cuh: large matrices; the
// context's stream, synchronised), records an event on the context's
// stream and returns: a host thread of its own builds the coarse levels
// from A_1, or else copies the matrix (on a stream of its own, after that
// event) and builds the whole hierarchy, and stages it.  The caller
// may issue more device work meanwhile; amg_build_end, on the caller's
// thread, waits for the host part, allocates and uploads (stream-ordered)
// and fills the outputs as amg_build does, frees the job and clears *job
// (errors of the host part are returned there, and also free the job).
// When only the device allocation fails (RBFFD_ENOMEM) the finished job is
// kept in *job, so the upload can be retried later without repeating the
// host part.  amg_build_abandon joins and frees a job that is not needed
// any more (NULL is allowed).  The packed matrix must not change until
// the host part has been joined by amg_build_end or amg_build_abandon.
struct AmgJob;
template <typename T>
int amg_build_begin(rbffd_ctx *ctx, int n, int q, int ldn, const int32_t *col,
                    const double *val, int nblocks, int wpb, AmgJob **job);
template <typename T>
int amg_build_end(rbffd_ctx *ctx, AmgJob **job, void **mem, size_t *bytes, void **mem0,
                  size_t *bytes0, const AmgDevT<T> **dev, AmgDevT<T> *host_view,
                  AmgInfo *info);
void amg_build_abandon(AmgJob *job);

}  // namespace rbffd

// batch_rt.cu - releases the batch cache of an expression object.
#include "fx/batch.cuh"

namespace fx {

void free_batch_cache(fx_expr* x) {
  if (!x || !x->batch) return;
  if (x->batch->cur.exec) cudaGraphExecDestroy(x->batch->cur.exec);
  x->batch->cur.dev.release();
  delete x->batch;
  x->batch = nullptr;
}

}  // namespace fx

// Aggregated image graphs (Sec. III-C): super-vertex basis and graph.
#include "rw_internal.cuh"

rw_status rw_aggregate(rw_graph* g, rw_basis* b, const rw_topology_update* u, cudaStream_t st,
                       rw_graph** gout, rw_basis** bout) {
  (void)g; (void)b; (void)u; (void)st; (void)gout; (void)bout;
  return RW_ERR_UNSUPPORTED;
}

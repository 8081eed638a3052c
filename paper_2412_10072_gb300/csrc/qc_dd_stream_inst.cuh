// qc_dd_stream_inst.cuh -- instantiations of the streaming kernel of chains with directions
// for one family of solved terms (included by qc_dd_stream_diag.cu, qc_dd_stream_full.cu
// and qc_dd_stream_delay.cu, compiled in parallel).
#pragma once
#include "qc_internal.h"

namespace qc_dds {
using namespace qc;

template <int GK, int OK, bool OLEFT, bool DSUMS>
cudaError_t launch(dim3 grid, int block, int smem_bytes, cudaStream_t st, const DDStreamArgs &a)
{
    dd_stream_kernel<GK, OK, OLEFT, DSUMS, DDS_DEPTH><<<grid, block, smem_bytes, st>>>(a);
    return cudaGetLastError();
}

template <int GK, int OK, bool OLEFT, bool DSUMS> DDSLaunch make()
{
    DDSLaunch l;
    l.fn = (const void *)dd_stream_kernel<GK, OK, OLEFT, DSUMS, DDS_DEPTH>;
    l.launch = launch<GK, OK, OLEFT, DSUMS>;
    return l;
}

template <int GK, bool DSUMS> DDSLaunch pick(int ok, bool oleft)
{
    if (ok == KIND_NONE) return make<GK, KIND_NONE, false, DSUMS>();
    if (ok == KIND_DIAG) return oleft ? make<GK, KIND_DIAG, true, DSUMS>() : make<GK, KIND_DIAG, false, DSUMS>();
    if (ok == KIND_FULL) return oleft ? make<GK, KIND_FULL, true, DSUMS>() : make<GK, KIND_FULL, false, DSUMS>();
    return DDSLaunch();
}
} // namespace qc_dds

// qc_dd_stream_inst.cuh -- instantiations of the streaming kernel of chains with directions
// for one family of solved terms (included by the qc_dd_stream_*.cu units, which compile in
// parallel).
#pragma once
#include "qc_internal.h"

namespace qc_dds {
using namespace qc;

template <int GK, int OK, bool OLEFT, bool DSUMS, int SD>
cudaError_t launch(dim3 grid, int block, int smem_bytes, cudaStream_t st, const DDStreamArgs &a)
{
    dd_stream_kernel<GK, OK, OLEFT, DSUMS, SD, DDS_DEPTH><<<grid, block, smem_bytes, st>>>(a);
    return cudaGetLastError();
}

template <int GK, int OK, bool OLEFT, bool DSUMS, int SD> DDSLaunch make()
{
    DDSLaunch l;
    l.fn = (const void *)dd_stream_kernel<GK, OK, OLEFT, DSUMS, SD, DDS_DEPTH>;
    l.launch = launch<GK, OK, OLEFT, DSUMS, SD>;
    l.dirs_per_cta = SD;
    return l;
}

template <int GK, bool DSUMS, int SD> DDSLaunch pick(int ok, bool oleft)
{
    if (ok == KIND_NONE) return make<GK, KIND_NONE, false, DSUMS, SD>();
    if (ok == KIND_DIAG) return oleft ? make<GK, KIND_DIAG, true, DSUMS, SD>() : make<GK, KIND_DIAG, false, DSUMS, SD>();
    if (ok == KIND_FULL) return oleft ? make<GK, KIND_FULL, true, DSUMS, SD>() : make<GK, KIND_FULL, false, DSUMS, SD>();
    return DDSLaunch();
}
} // namespace qc_dds

// qc_dd_stream_diag.cu -- streaming kernels of chains with directions: direction-independent diagonal solved terms.
#include "qc_dd_stream_inst.cuh"

DDSLaunch dds_launcher_diag(int ok, bool oleft) { return qc_dds::pick<qc::KIND_DIAG, false, 0>(ok, oleft); }

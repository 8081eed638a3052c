// qc_dd_stream_full.cu -- streaming kernels of chains with directions: direction-independent full-Jones solved terms.
#include "qc_dd_stream_inst.cuh"

DDSLaunch dds_launcher_full(int ok, bool oleft) { return qc_dds::pick<qc::KIND_FULL, false, 0>(ok, oleft); }

// qc_dd_stream_full_dd.cu -- streaming kernels of chains with directions: direction-dependent full-Jones solved terms, one direction per CTA.
#include "qc_dd_stream_inst.cuh"

DDSLaunch dds_launcher_full_dd(int ok, bool oleft) { return qc_dds::pick<qc::KIND_FULL, false, 1>(ok, oleft); }

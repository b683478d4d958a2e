"""Measurement probes (not part of the library): int_pipes.cu measures the
integer-pipe throughput the sweep kernels are bound by.

    python -m paper_2404_16990_gb300.probes
"""

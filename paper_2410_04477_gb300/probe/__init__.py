"""Arithmetic-pipe throughput probe for the ALU rooflines (run on the GPU):
``python -m paper_2410_04477_gb300.probe`` prints FP64 and FP32 FMA rates, full warps and
single active lanes."""

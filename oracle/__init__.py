"""FP64 CPU oracle for the two-component Shan-Chen D3Q19 LB with suspended
spheres (arXiv:1004.4414).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product package.
"""

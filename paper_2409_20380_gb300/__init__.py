"""GB300-native matrix-free EBE solver for many time-evolution linear-elastic FE cases with a
data-driven initial-guess predictor (arXiv 2409.20380).  The compute path is libfem.so (include/fem.h);
`fem` is its Python binding and `workload` generates the seeded synthetic inputs."""

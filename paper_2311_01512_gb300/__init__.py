"""GB300-native local full-state quantum simulation (statevectors and density
matrices as Choi vectors), after arXiv 2311.01512.

The CUDA library is loaded by ``paper_2311_01512_gb300.qs``; importing the
package itself does not load it, so that ``workloads`` stays usable on hosts
without a GPU.
"""

"""GB300-native sampled-gradient GCP (GCP-SGD / GCP-Adam, arXiv:1906.01687).

The compute path is the CUDA library ``libgcp_gb300.so`` (sources in
``csrc/``, C ABI in ``include/gcp.h``).  ``paper_1906_01687_gb300.gcp`` is its
thin ctypes binding; importing it loads the library and raises if it has not
been built.  ``paper_1906_01687_gb300.synth`` makes seeded synthetic inputs
and loads nothing.  This file imports neither, so that importing one does
not pull in the other.
"""

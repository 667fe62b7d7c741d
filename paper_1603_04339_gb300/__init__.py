"""GB300-native CheFSI hot path of real-space Kohn-Sham DFT (SPARC, arXiv:1603.04339).

The compute lives in the C-ABI library ``libsparc.so`` (CUDA, sm_103a); the
Python modules here only build it and marshal arguments to it.  Importing the
package does not load the library: ``paper_1603_04339_gb300.sparc`` does.
"""

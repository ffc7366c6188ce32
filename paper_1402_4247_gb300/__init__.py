"""GB300-native band step of numerical-atomic-orbital DFT (Band_DFT_Col, arXiv:1402.4247 Sec. 3).

The compute path is the CUDA library ``libnao.so`` behind the C ABI in ``include/nao.h``;
``paper_1402_4247_gb300.nao`` is its Python binding and ``paper_1402_4247_gb300.synth``
makes seeded synthetic inputs.  Submodules are imported explicitly, so the input
generator works on machines without a GPU or torch.
"""

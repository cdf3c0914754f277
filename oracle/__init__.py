"""Oracle for the FFT stencil path: plain, slow, obviously correct, CPU, FP64.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import or call anything in
this package. The product path (``paper_2105_06676_gb300``) never imports it,
and this package imports nothing from the product path: the two share no
kernels, headers, helpers, tables or constants. The only thing both sides
consume is the seeded input generator module, which holds none of the method's
arithmetic.

Contents
--------
``stencil_loop``         the plain definition a_{t+1} = S a_t written out as a
                         double-buffered nested loop in C (periodic and
                         zero-Dirichlet), compiled with gcc. Paper Sec. 1
                         "Problem Specification" and the looping codes of
                         Fig. "looping-code".
``spectral``             the paper's StencilFFT-P steps in numpy FP64 (first
                         column of S, Multi-FFT, repeated squaring, pointwise
                         product, inverse Multi-FFT), Sec. 4 and
                         Fig. "stencil-fft-algorithm-dD"; closed-form symbol,
                         Appendix "Proof of Eigenvalue-FFT Relation".
``recursive_boundary``   StencilFFT-A and RecursiveBoundary in numpy FP64,
                         Sec. 5 and Fig. "stencil-fft-algorithm-1D-aperiodic"
                         (zero-Dirichlet or reflecting base case).
``ell_shells``           RecursiveBoundary with its regions in l-shells (the
                         step at which the boundary's influence reaches a
                         cell, per-face reach of biased stencils), appendix
                         "l-shell Spatial Grid Decomposition".
``implicit``             implicit stencils Q a_{t+1} = S a_t: dense
                         pseudoinverse definition and the spectral method with
                         Lambda_R = Lambda_Q^+ Lambda_S, appendix "Supporting
                         Implicit Stencils".
``vector_fields``        vector-valued fields: the plain m-field loop and the
                         spectral method with a matrix of symbols raised by
                         repeated squaring, appendix "Supporting Vector Valued
                         Fields".

Every function is pinned by ``tests/test_oracle_pins.py`` against values the
paper prints, closed forms, invariants and brute force.
"""
from .stencil_loop import (  # noqa: F401
    build_oracle_library,
    oracle_library_path,
    oracle_threads,
    stencil_loop,
)
from .spectral import (  # noqa: F401
    dft_naive,
    first_column,
    stencil_fft_periodic,
    symbol_closed_form,
    symbol_multi_fft,
    symbol_power,
)
from .recursive_boundary import (  # noqa: F401
    boundary_distance,
    recursive_boundary,
    stencil_fft_aperiodic,
)
from .ell_shells import (  # noqa: F401
    arrival_time,
    face_distances,
    face_reach,
    recursive_boundary_shells,
    stencil_fft_aperiodic_shells,
)
from .implicit import (  # noqa: F401
    implicit_dense,
    implicit_symbol,
    stencil_fft_periodic_implicit,
    stencil_matrix,
    zero_threshold,
)
from .vector_fields import (  # noqa: F401
    matrix_power_sq,
    stencil_fft_periodic_vector,
    symbol_matrix,
    vector_loop,
)

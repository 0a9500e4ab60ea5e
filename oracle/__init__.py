"""FP64 CPU oracle for TAN(-SIP) reprojection — TEST INFRASTRUCTURE, not part of the product.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The product library never calls it, and it shares no code with the CUDA
path: every formula here is restated from the paper (dfreproject, arXiv 2505.03932) and the
standards it cites (Greisen & Calabretta 2002, Calabretta & Greisen 2002, Shupe et al. 2005).

Modules
    wcs      pixel -> world (Sec. 3.2.1) and world -> pixel (Sec. 3.2.2), SIP polynomials,
             the inverse-SIP least-squares fit, the exact (Newton) SIP inverse, and an
             independent FITS header parser.
    interp   nearest / bilinear / bicubic (Keys) interpolation with the footprint
             normalisation of Sec. 3.1, and its adjoint (transpose).
    reproject  the whole per-pixel map (Sec. 3.1 steps 1-3) over a target grid or a pixel
             sample.
    dual     forward-mode dual numbers; gradients of a reprojection loss with respect to the
             source WCS parameters.

Parity status: every function is pinned by a CPU test (tests/test_oracle_*.py) against a
closed form, an invariant, a library routine or brute force; none is "parity unpinned" except
the SIP sign convention, whose pin is the definition in Shupe et al. (2005) (a hand-worked
golden case), not an external implementation.
"""

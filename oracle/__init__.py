"""CPU oracle for recycled mixed-precision GMRES-IR (RGMRES-IR).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package. The product (the CUDA library and its Python binding)
never calls it, and this package never imports the product.

Plain, slow, FP64 / double-double numpy code that follows the paper's algorithms
step by step:

* ``formats``   -- rounding to fp16 / bf16 / fp32 / fp8-e4m3 (unit roundoffs of Table 1).
* ``dd``        -- double-double arithmetic (stands in for the paper's quad precision).
* ``lu``        -- LU with partial pivoting in precision u_f (Algorithm 4, the factorization step), in the
                   paper's "every operation rounded" form and in the block-FMA form
                   (u_f operands, FP32 accumulation) that tensor cores implement.
* ``gcrodr``    -- GCRO-DR(m, k) (Algorithm 3) including the harmonic-Ritz recycle update.
* ``ir``        -- GMRES-IR / RGMRES-IR (Algorithms 2 and 4), the adjoint solve and batches.

Parity status of each function is stated in its docstring; "parity unpinned"
marks the ones no test ties to something other than the oracle itself.
"""

"""GB300-native exact polynomial-matrix arithmetic over F_p (libpmat).

The product A(x).B(x) mod p in full, truncated and middle-product form (also from and to host
memory), the PM-Basis approximant basis and the PM-IntBasis interpolant basis built on it, the
bivariate resultant (direct method and Villard variant), the truncated inverse A^-1 mod x^t, the
series solution A^-1 b mod x^N (by Dixon's or by high-order lifting), the lifting solver
A u = f b and the high-order lifting slices, all behind the C ABI in include/pmat.h; ``pmat`` is
its Python binding.
"""
from .pmat import (Context, PmError, bivariate_resultant, bivariate_resultant_villard, lib, pm_basis, pm_intbasis,
                   pmat_inv_slices, pmat_inv_trunc, pmat_middle_product, pmat_mul, pmat_mul_batched, pmat_mul_host,
                   pmat_mul_trunc, pmat_solve, pmat_solve_series, pmat_solve_series_hol, to_device, to_host)

__all__ = ["Context", "PmError", "lib", "pmat_mul", "pmat_mul_trunc", "pmat_middle_product", "pmat_mul_host",
           "pmat_mul_batched", "pmat_inv_trunc", "pmat_solve_series", "pmat_solve_series_hol", "pmat_solve",
           "pmat_inv_slices", "pm_basis", "pm_intbasis", "bivariate_resultant", "bivariate_resultant_villard",
           "to_device", "to_host"]

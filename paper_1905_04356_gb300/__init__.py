"""GB300-native exact polynomial-matrix arithmetic over F_p (libpmat).

The product A(x).B(x) mod p in full, truncated and middle-product form, the
PM-Basis approximant basis built on it, the bivariate resultant and the
truncated inverse A^-1 mod x^t and the lifted series solution A^-1 b mod
x^N, all behind the C ABI in include/pmat.h;
``pmat`` is its Python binding.
"""
from .pmat import (Context, PmError, bivariate_resultant, lib, pm_basis, pmat_middle_product, pmat_mul,
                   pmat_inv_slices, pmat_inv_trunc, pmat_mul_batched, pmat_mul_trunc, pmat_solve_series, to_device,
                   to_host)

__all__ = ["Context", "PmError", "lib", "pmat_mul", "pmat_mul_trunc", "pmat_middle_product", "pmat_inv_trunc", "pmat_solve_series", "pmat_inv_slices",
           "pmat_mul_batched", "pm_basis", "bivariate_resultant", "to_device", "to_host"]

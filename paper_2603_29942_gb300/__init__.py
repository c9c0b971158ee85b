"""GB300-native certified minimum distance of linear codes over F_p.

The Brouwer-Zimmermann enumeration (arXiv 2603.29942, Sec. 3.1) runs as a
persistent sm_103a CUDA kernel behind the C ABI in include/fpcode.h; this
package is its thin Python binding (``_binding``), the in-tree build
(``build``) and the seeded workload generators (``inputs``).
"""
from . import inputs  # noqa: F401

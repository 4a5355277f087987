"""GB300-native grid hopping (range-Doppler maps, hopping scorer, argmax, BOMP
and the exact direct decision function) behind a C-ABI CUDA library.

``gh`` is the thin binding over ``libgh.so``; ``scenes`` makes seeded
synthetic inputs. The binding loads the library on first use and raises if it
is missing: there is no CPU fallback.
"""

"""GB300-native (sm_103a) ICNNM: tensor completion with pre-learned convolution
eigenvectors (arxiv 2604.17001). The compute path is libicnnm.so (hand-written CUDA,
C ABI in include/icnnm.h); ``icnnm`` is its thin ctypes binding. Importing the
package loads nothing; ``synth`` holds the seeded input generators."""

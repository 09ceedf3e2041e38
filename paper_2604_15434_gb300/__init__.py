"""GB300-native screened EFTofDE particle-mesh library (placeholder while the binding is built)."""
